// Persistent bound-propagation engine (Section 2.1) for sm_103a.
//
// One cooperative launch runs a whole propagation: a prologue that normalises the caller's
// bounds, one phase per Jacobi round, and an epilogue that writes the bounds back.  A phase
// processes the round's worklist of rows:
//   minimal activity  L_min = sum_{a>0} a l + sum_{a<0} a u  (finite part + count of infinite
//                     terms), one fused multiply-add per nonzero;
//   row verdict       infeasible if no infinite term and L_min > g + tol;
//   candidates        u_i <= (g - L_min + a l_i) / a (a > 0), l_i >= (g - L_min + a u_i) / a
//                     (a < 0), after an FP32 prefilter that proves most of them cannot tighten;
//   apply             atomicMin / atomicMax of ordered keys into the next round's bounds; the
//                     first change of a variable in the round queues its rows for the next
//                     round ("propagation on changed constraints", Section 1).
// Rounds are separated by one grid barrier.  All waits are bounded: a wait that runs out sets
// BP_ERR_TIMEOUT and the launch returns.
//
// The rounds are latency-bound (a round is a chain of dependent L2 round trips and of
// synchronising operations, each a few hundred cycles on GB300), so all work of a round is
// warp-sized and spread over every SM, and a round holds as few synchronising steps as
// possible:
//   phase A   warp tasks [pieces][fix-ups of the previous round's changes][thread-per-row
//             bins][warp rows]: short rows are finished here (activity, verdict, candidates);
//             a piece (a slice of at most kPieceMax nonzeros of a long row) stores its partial
//             activity in its slot;
//   barrier   only when the round has pieces;
//   phase B   every piece sums its row's partials in slot order (the same order for every piece
//             of the row, so all see the same total), the first piece records the row's verdict
//             and work, and each piece evaluates its own nonzeros' candidates;
//   then the changed variables are listed and their rows queued for the next round, and the
//   round ends at the grid barrier.  No task ever waits for another task.
#include <climits>
#include <cstdlib>

#include "bp_host.h"
#include "fp_draw.cuh"

namespace gpubp {

#ifndef GPUBP_MIN_BLOCKS
#define GPUBP_MIN_BLOCKS 2     // resident blocks per SM the register budget is sized for
#endif

constexpr int kThreads = 256;
constexpr int kWarpsPerBlock = kThreads / 32;
constexpr int kSlots = kNumClass;               // staging slots: row classes 0..5, then changed vars
constexpr int kSlotChg = kClassPieces;          // piece rows are not staged; their slot holds variables
constexpr int kBq = 2048;                       // per-block queue of accepted variables
constexpr int kMaxInst = kMaxInstances;         // instances per batched launch
constexpr long long kSpinLimit = 4000000000LL;  // clock64 cycles (about 2 s) per wait
static_assert(32 * kPerThread == kPieceMax, "the longest piece is one wave of a warp");

struct BpArgs {
    double* lb;
    double* ub;
    longlong2* bk[2];
    int* vstamp;
    int* rstamp;
    int* list[2];
    int* chg[2];
    int4* task[2];
    double* hpart;
    int2* hpinf;
    Ctl* ctl;
    bp_result* dres;
    const int* w0;      // rows of round 0, or null for every row
    int w0_len;
    const int* w0v;     // or: variables whose rows form round 0 (count in *w0v_len)
    const int* w0v_len;
    double theta;
    int max_rounds;
    int* stamp;         // device word: stamp of round 0, advanced at exit (graph replays stay valid)
    long long* trace;   // optional: 4 words per round
    // instances: a batch of independent problems laid out block-diagonally (rows
    // [row_off[i], row_off[i+1]) and variables [col_off[i], col_off[i+1]) form instance i).
    // One instance (ninst = 1, null offsets) is a plain propagation.
    int skip_block;     // test only (GPUBP_TEST_SKIP_BLOCK): this block leaves without arriving, -1 none
    int ninst;
    const int* row_off;
    const int* col_off;
    InstState* inst;
    // optional (device-driven rounding loop): every variable changed during the propagation is
    // listed once in dirty[0 .. *ndirty), deduplicated by vdirty[v] == the block's dstamp
    int* vdirty;
    int* dirty;
    int* ndirty;
    unsigned long long* i_nnz;   // [kPhaseSlots][ninst] nonzeros processed in the round of that slot
    int* i_rowinf;               // [kPhaseSlots][ninst] smallest infeasible row of the round
    int* i_cross;                // [kPhaseSlots][ninst] smallest crossing variable found in the round
    int* i_chg;                  // [kPhaseSlots][ninst] a variable of the instance changed in the round
};

__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

struct Stage {
    int wcnt[kWarpsPerBlock][kSlots];           // per-warp private staging of appends
    int wbuf[kWarpsPerBlock][kSlots][32];
    int bq_n;                                   // variables with an accepted candidate in this phase
    int bq[kBq];
    unsigned long long nnz;
    int flag;
    // descriptor of the current phase, read once per block by thread 0
    int d_cnt[kNumClass];
    int d_ntask, d_nprev;
    // instances (offsets; live and pending-check flags and result buffer, kept by every block
    // from the same verdicts)
    int roff[kMaxInst + 1], coff[kMaxInst + 1];
    unsigned char alive[kMaxInst], pending[kMaxInst], rpar[kMaxInst];
    unsigned long long i_nnz[kMaxInst];
    int any_alive;
    int last_block;
    unsigned bar_k;                              // grid barriers passed in this launch
    int epi_n, epi_par;                          // variables changed in the last round, their list
    int dstamp;                                  // stamp of the current propagation in vdirty
    int go;                                      // block-uniform decision of a device-driven loop
};

// ------------------------------------------------------------------ phase state
struct Phase {
    int t, par, npar;
    // counter slots of this round and of the next
    __device__ __forceinline__ int s3() const { return t % kPhaseSlots; }
    __device__ __forceinline__ int ns3() const { return (t + 1) % kPhaseSlots; }
    const longlong2* R;     // bounds at the start of the round
    longlong2* X;           // bounds of the next round (atomics)
    int st_v, st_r;         // variable-change stamp of this round, row stamp of next round
};

// instance of row k / variable v (binary search in the shared-memory offsets)
__device__ __forceinline__ int find_inst(const int* off, int ninst, int x) {
    int lo = 0, hi = ninst - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= x) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}
__device__ __forceinline__ int row_inst(const Stage& st, const BpArgs& A, int k) {
    return A.ninst == 1 ? 0 : find_inst(st.roff, A.ninst, k);
}
__device__ __forceinline__ int var_inst(const Stage& st, const BpArgs& A, int v) {
    return A.ninst == 1 ? 0 : find_inst(st.coff, A.ninst, v);
}

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Global destination and counter of staging slot s.
__device__ __forceinline__ int* slot_dst(const BpArgs& A, const DevProblem& P, const Phase& ph, int s, int pos) {
    return s == kSlotChg ? A.chg[ph.par] + pos : A.list[ph.npar] + P.class_off[s] + pos;
}
__device__ __forceinline__ int* slot_ctr(const BpArgs& A, const Phase& ph, int s) {
    return s == kSlotChg ? &A.ctl->nchg[ph.s3()].v : &A.ctl->cnt[ph.ns3()][s].v;
}

// Warp-wide: move this warp's staged entries of slot s to the global list (one atomic).
__device__ __forceinline__ void warp_flush_slot(Stage& st, const BpArgs& A, const DevProblem& P, const Phase& ph,
                                                int s) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncwarp();
    const int n = st.wcnt[w][s];
    if (n == 0) return;
    int base = 0;
    if (lane == 0) base = atomicAdd(slot_ctr(A, ph, s), n);
    base = __shfl_sync(0xffffffffu, base, 0);
    if (lane < n) *slot_dst(A, P, ph, s, base + lane) = st.wbuf[w][s][lane];
    __syncwarp();
    if (lane == 0) st.wcnt[w][s] = 0;
    __syncwarp();
}

__device__ void warp_flush_all(Stage& st, const BpArgs& A, const DevProblem& P, const Phase& ph) {
    for (int s = 0; s < kSlots; ++s) warp_flush_slot(st, A, P, ph, s);
}

// Warp-wide (all 32 lanes, converged): append `value` to staging slot `slot` for every lane
// with slot >= 0.  Lanes with equal slots share one staging update; a full slot is flushed
// with one global atomic for up to 32 entries.
__device__ void warp_append(Stage& st, const BpArgs& A, const DevProblem& P, const Phase& ph, int slot, int value) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    unsigned pending = __ballot_sync(0xffffffffu, slot >= 0);
    while (pending) {
        const int src = __ffs(pending) - 1;
        const int s = __shfl_sync(0xffffffffu, slot, src);
        const unsigned grp = __ballot_sync(0xffffffffu, slot == s) & pending;
        const int n = __popc(grp);
        __syncwarp();
        int cnt = st.wcnt[w][s];
        if (cnt + n > 32) {
            warp_flush_slot(st, A, P, ph, s);
            cnt = 0;
        }
        if (grp & (1u << lane)) st.wbuf[w][s][cnt + __popc(grp & lanemask_lt())] = value;
        __syncwarp();
        if (lane == 0) st.wcnt[w][s] = cnt + n;
        __syncwarp();
        pending &= ~grp;
    }
}

// Append of one row or variable by a single lane, straight to the global lists (only for the
// rare paths that run outside a converged warp).
__device__ void lane_queue_row(const BpArgs& A, const DevProblem& P, const Phase& ph, int k) {
    const int info = __ldg(P.rinfo + k);   // issued before the stamp atomic: no dependency
    const int rb = __ldg(P.row_ptr + k), re = __ldg(P.row_ptr + k + 1);
    if (atomicMax(&A.rstamp[k], ph.st_r) >= ph.st_r) return;
    const int cls = info & 7;
    if (cls != kClassPieces) {
        const int pos = atomicAdd(&A.ctl->cnt[ph.ns3()][cls].v, 1);
        A.list[ph.npar][P.class_off[cls] + pos] = k;
        return;
    }
    const int nch = info >> 3;
    const int base = atomicAdd(&A.ctl->ntask[ph.ns3()].v, nch);
    for (int c = 0; c < nch; ++c) A.task[ph.npar][base + c] = piece_desc(k, c, rb, re, P.chunk_len);
    atomicAdd(&A.ctl->cnt[ph.ns3()][kClassPieces].v, 1);
}

// Warp-wide: queue the rows `k` (k < 0: none) for the next round; a row's first queuing in
// this round wins.  A piece row gets its pieces, contiguous and in row order, in the piece list
// (the lanes with piece rows write them together).
__device__ void warp_queue_rows(Stage& st, const BpArgs& A, const DevProblem& P, const Phase& ph, int k) {
    const int lane = threadIdx.x & 31;
    int slot = -1, nch = 0, base = 0;
    // issued before the stamp atomic (no dependency): class, pieces and the row's extent
    const int info = k >= 0 ? __ldg(P.rinfo + k) : 0;
    const int rb = k >= 0 ? __ldg(P.row_ptr + k) : 0, re = k >= 0 ? __ldg(P.row_ptr + k + 1) : 0;
    if (k >= 0 && atomicMax(&A.rstamp[k], ph.st_r) < ph.st_r) {
        const int cls = info & 7;
        if (cls != kClassPieces) {
            slot = cls;
        } else {
            nch = info >> 3;
            base = atomicAdd(&A.ctl->ntask[ph.ns3()].v, nch);
            atomicAdd(&A.ctl->cnt[ph.ns3()][kClassPieces].v, 1);
        }
    }
    unsigned longs = __ballot_sync(0xffffffffu, nch > 0);
    while (longs) {
        const int src = __ffs(longs) - 1;
        const int kk = __shfl_sync(0xffffffffu, k, src);
        const int nn = __shfl_sync(0xffffffffu, nch, src);
        const int bb = __shfl_sync(0xffffffffu, base, src);
        const int rbb = __shfl_sync(0xffffffffu, rb, src), ree = __shfl_sync(0xffffffffu, re, src);
        for (int c = lane; c < nn; c += 32) A.task[ph.npar][bb + c] = piece_desc(kk, c, rbb, ree, P.chunk_len);
        longs &= longs - 1;
    }
    warp_append(st, A, P, ph, slot, k);
}

// Variable j had a candidate accepted in this round: remember it in the block's queue (shared
// memory only; no global round trip on the task's path).  drain_changed later keeps the first
// report of each variable across the grid and queues its rows.  A full queue falls back to
// doing that work from this lane.
// Lists variable v once per propagation in the dirty list (device-driven rounding loop only).
__device__ __noinline__ void note_dirty(const BpArgs& A, int stamp, int v) {
    if (atomicMax(&A.vdirty[v], stamp) < stamp) A.dirty[atomicAdd(A.ndirty, 1)] = v;
}

__device__ __forceinline__ void note_changed(Stage& st, const BpArgs& A, const DevProblem& P, const Phase& ph,
                                             int j) {
    const int i = atomicAdd(&st.bq_n, 1);
    if (i < kBq) {
        st.bq[i] = j;
        return;
    }
    if (atomicMax(&A.vstamp[j], ph.st_v) >= ph.st_v) return;
    A.i_chg[ph.s3() * A.ninst + var_inst(st, A, j)] = 1;
    if (A.vdirty) note_dirty(A, st.dstamp, j);
    const int pos = atomicAdd(&A.ctl->nchg[ph.s3()].v, 1);
    A.chg[ph.par][pos] = j;
    const int e = __ldg(P.col_ptr + j + 1);
    for (int s = __ldg(P.col_ptr + j); s < e; ++s) lane_queue_row(A, P, ph, __ldg(P.row_idx + s));
}

// Block-wide, once per phase: for every variable in the block's queue that changes for the
// first time in this round (grid-wide), list it and queue its rows.  Each warp takes 32
// variables at a time and spreads their (variable, row) pairs over its lanes, so a batch of
// columns costs a few round trips in total.
__device__ void drain_changed(Stage& st, const BpArgs& A, const DevProblem& P, const Phase& ph) {
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int n = min(st.bq_n, kBq);
    for (int b0 = w * 32; b0 < n; b0 += kThreads) {
        const int idx = b0 + lane;
        int v = idx < n ? st.bq[idx] : -1;
        // the column extent is loaded alongside the stamp atomic (independent round trips)
        const int cb = v >= 0 ? __ldg(P.col_ptr + v) : 0;
        const int ce = v >= 0 ? __ldg(P.col_ptr + v + 1) : 0;
        if (v >= 0 && atomicMax(&A.vstamp[v], ph.st_v) >= ph.st_v) v = -1;
        if (v >= 0) A.i_chg[ph.s3() * A.ninst + var_inst(st, A, v)] = 1;
        if (A.vdirty && v >= 0) note_dirty(A, st.dstamp, v);
        warp_append(st, A, P, ph, v >= 0 ? kSlotChg : -1, v);
        const int deg = v >= 0 ? ce - cb : 0;
        int incl = deg;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        const int excl = incl - deg;
        const int total = __shfl_sync(0xffffffffu, incl, 31);
        for (int p0 = 0; p0 < total; p0 += 32) {
            const int p = p0 + lane;
            // owner lane: the last lane whose exclusive offset is <= p
            int owner = 0;
            for (int step = 16; step >= 1; step >>= 1) {
                const int e = __shfl_sync(0xffffffffu, excl, owner + step);
                if (e <= p) owner += step;
            }
            const int ob = __shfl_sync(0xffffffffu, cb, owner);
            const int oe = __shfl_sync(0xffffffffu, excl, owner);
            const int k = p < total ? __ldg(P.row_idx + ob + (p - oe)) : -1;
            warp_queue_rows(st, A, P, ph, k);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) st.bq_n = 0;
    __syncthreads();
}

// Exact candidate of variable j (see eval_candidate) and its application: atomicMin / atomicMax
// of the new key into the next round's bounds, and a note in the block's change queue.
__device__ __forceinline__ void try_candidate(Stage& st, const BpArgs& A, const DevProblem& P, const Phase& ph,
                                              double a, int j, longlong2 bk, double minfin, int ninf, double g) {
    long long nk;
    const int r = eval_candidate(a, bk.x, bk.y, minfin, ninf, g, P.is_int[j] != 0, A.theta, &nk);
    if (r == 1) {
        atomicMin(&ph.X[j].y, nk);
        note_changed(st, A, P, ph, j);
    } else if (r == 2) {
        atomicMax(&ph.X[j].x, nk);
        note_changed(st, A, P, ph, j);
    }
}

struct Acc {
    double minfin;
    int ninf, infj;
};

__device__ __forceinline__ Acc warp_reduce(Acc a) {
    for (int off = 16; off > 0; off >>= 1) {
        a.minfin = __dadd_rn(a.minfin, __shfl_xor_sync(0xffffffffu, a.minfin, off));
        a.ninf += __shfl_xor_sync(0xffffffffu, a.ninf, off);
        a.infj = max(a.infj, __shfl_xor_sync(0xffffffffu, a.infj, off));
    }
    return a;
}

// A thread's share of a row range: at most kPerThread nonzeros, held in registers.
struct Elems {
    int j[kPerThread];
    double a[kPerThread];
    longlong2 bk[kPerThread];
};

// Loads the nonzeros beg + tid + i*stride (i < kPerThread, < end) in one wave, gathers their
// bounds in a second wave, and accumulates the thread's part of the minimal activity.
__device__ __forceinline__ Acc load_accumulate(Elems& E, const DevProblem& P, const Phase& ph, int beg, int end,
                                               int tid, int stride) {
#pragma unroll
    for (int i = 0; i < kPerThread; ++i) {
        const int q = beg + tid + i * stride;
        E.j[i] = q < end ? __ldg(P.col + q) : -1;
        E.a[i] = q < end ? __ldg(P.val + q) : 0.0;
    }
#pragma unroll
    for (int i = 0; i < kPerThread; ++i) E.bk[i] = E.j[i] >= 0 ? ld_bounds(ph.R, E.j[i]) : make_longlong2(0, 0);
    Acc s{0.0, 0, -1};
#pragma unroll
    for (int i = 0; i < kPerThread; ++i) {
        if (E.j[i] < 0) continue;
        const long long key = E.a[i] > 0 ? E.bk[i].x : E.bk[i].y;
        if (key_is_inf(key)) {
            ++s.ninf;
            s.infj = E.j[i];
        } else {
            s.minfin = fma(E.a[i], kdec(key), s.minfin);
        }
    }
    return s;
}

// The loads of load_accumulate without the sum (the candidate pass of a piece).
__device__ __forceinline__ void load_elems(Elems& E, const DevProblem& P, const Phase& ph, int beg, int end, int tid,
                                           int stride) {
#pragma unroll
    for (int i = 0; i < kPerThread; ++i) {
        const int q = beg + tid + i * stride;
        E.j[i] = q < end ? __ldg(P.col + q) : -1;
        E.a[i] = q < end ? __ldg(P.val + q) : 0.0;
    }
#pragma unroll
    for (int i = 0; i < kPerThread; ++i) E.bk[i] = E.j[i] >= 0 ? ld_bounds(ph.R, E.j[i]) : make_longlong2(0, 0);
}

// Elements of E that may tighten a bound given the row total (bit i for element i): with one
// infinite term only that term's variable (no prefilter), with none every element the FP32
// prefilter cannot rule out.
__device__ __forceinline__ unsigned elems_pass(const Elems& E, const Acc& tot, double g) {
    unsigned pass = 0;
    if (tot.ninf >= 2) return 0;
    if (tot.ninf == 1) {
#pragma unroll
        for (int i = 0; i < kPerThread; ++i)
            if (E.j[i] >= 0 && E.j[i] == tot.infj) pass |= 1u << i;
        return pass;
    }
    const RowFilter f = row_filter(g, tot.minfin);
#pragma unroll
    for (int i = 0; i < kPerThread; ++i)
        if (E.j[i] >= 0 && !cannot_tighten(f, E.a[i], E.bk[i].x, E.bk[i].y)) pass |= 1u << i;
    return pass;
}

// Exact evaluation and application of the elements of E whose bit is set in `pass`, with the
// lane's row data (finite activity, one-infinite-term flag, g).
__device__ __forceinline__ void eval_pass(Stage& st, const BpArgs& A, const DevProblem& P, const Phase& ph,
                                          const Elems& E, unsigned pass, double minfin, bool inf1, double g) {
    if (!pass) return;
#pragma unroll
    for (int i = 0; i < kPerThread; ++i)
        if (pass & (1u << i)) try_candidate(st, A, P, ph, E.a[i], E.j[i], E.bk[i], minfin, inf1 ? 1 : 0, g);
}

// The candidates of the thread's elements given the row total.
__device__ __forceinline__ void elems_candidates(Stage& st, const BpArgs& A, const DevProblem& P, const Phase& ph,
                                                 const Elems& E, const Acc& tot, double g) {
    eval_pass(st, A, P, ph, E, elems_pass(E, tot, g), tot.minfin, tot.ninf == 1, g);
}

// ------------------------------------------------------------------- row kernels
// Thread per row (rows of at most kThreadMax nonzeros): 32 rows per warp task.
__device__ void do_thread_rows(Stage& st, const BpArgs& A, const DevProblem& P, const Phase& ph,
                               const int* rows, int count, int tl) {
    const int idx = tl * 32 + (threadIdx.x & 31);
    const int k = idx < count ? __ldcg(rows + idx) : -1;
    const int ki = k >= 0 ? row_inst(st, A, k) : 0;
    if (k >= 0 && st.alive[ki]) {
        const int beg = __ldg(P.row_ptr + k), end = __ldg(P.row_ptr + k + 1);
        const double2 g2 = __ldg(P.grow + k);
        Elems E;
        const Acc s = load_accumulate(E, P, ph, beg, end, 0, 1);
        atomicAdd(&st.nnz, (unsigned long long)(end - beg));
        atomicAdd(&st.i_nnz[ki], (unsigned long long)(end - beg));
        if (row_infeasible(s.minfin, s.ninf, g2.y)) {
            atomicMin(&A.i_rowinf[ph.s3() * A.ninst + ki], k);
        } else {
            elems_candidates(st, A, P, ph, E, s, g2.x);
        }
    }
}

// Warp per row (kThreadMax+1 .. kWarpMax nonzeros).
__device__ void do_warp_row(Stage& st, const BpArgs& A, const DevProblem& P, const Phase& ph, int k) {
    const int lane = threadIdx.x & 31;
    const int ki = row_inst(st, A, k);
    if (!st.alive[ki]) return;
    const int beg = __ldg(P.row_ptr + k), end = __ldg(P.row_ptr + k + 1);
    const double2 g2 = __ldg(P.grow + k);
    Elems E;
    const Acc tot = warp_reduce(load_accumulate(E, P, ph, beg, end, lane, 32));
    if (lane == 0) {
        atomicAdd(&st.nnz, (unsigned long long)(end - beg));
        atomicAdd(&st.i_nnz[ki], (unsigned long long)(end - beg));
    }
    if (row_infeasible(tot.minfin, tot.ninf, g2.y)) {
        if (lane == 0) atomicMin(&A.i_rowinf[ph.s3() * A.ninst + ki], k);
    } else {
        elems_candidates(st, A, P, ph, E, tot, g2.x);
    }
}

// Bounds of a piece's nonzeros kept in registers from phase A to phase B: the gather is the
// dependent half of loading a piece, so phase B then only reissues the independent column and
// coefficient loads, together with the loads of the row's partials.
struct HeldBounds {
    longlong2 bk[kPerThread];
};

// Piece u of a piece row (descriptor tk, see piece_desc), phase A: the partial activity of its
// nonzeros into slot u; H (if given) keeps their bounds.
__device__ __forceinline__ void piece_partial(const BpArgs& A, const DevProblem& P, const Phase& ph, int u, int4 tk,
                                              HeldBounds* H) {
    const int lane = threadIdx.x & 31;
    const int beg = tk.z, end = min(tk.w, beg + P.chunk_len);
    Elems E;
    const Acc s = warp_reduce(load_accumulate(E, P, ph, beg, end, lane, 32));
    if (H) {
#pragma unroll
        for (int i = 0; i < kPerThread; ++i) H->bk[i] = E.bk[i];
    }
    if (lane == 0) {
        A.hpart[u] = s.minfin;
        A.hpinf[u] = make_int2(s.ninf, s.infj);
    }
}

// Piece u, phase B: the row total is the sum of the row's piece partials in slot order (the
// row's pieces sit in the consecutive slots u - c ..); every piece of the row computes it in the
// same order and gets the same value.  The first piece records the row's verdict and its
// nonzeros; each piece then evaluates its own nonzeros' candidates, with the bounds kept in H
// since phase A when given, else reloaded (L2).
__device__ __forceinline__ void piece_candidates(Stage& st, const BpArgs& A, const DevProblem& P, const Phase& ph,
                                                 int u, int4 tk, const HeldBounds* H) {
    const int lane = threadIdx.x & 31;
    const int k = tk.x, c = tk.y, beg = tk.z, re = tk.w;
    const int end = min(re, beg + P.chunk_len);
    const int ki = row_inst(st, A, k);
    const int npc = c + (re - beg + P.chunk_len - 1) / P.chunk_len;
    Elems E;
    if (H) {
        // issued with the partials' loads below (independent)
#pragma unroll
        for (int i = 0; i < kPerThread; ++i) {
            const int q = beg + lane + i * 32;
            E.j[i] = q < end ? __ldg(P.col + q) : -1;
            E.a[i] = q < end ? __ldg(P.val + q) : 0.0;
            E.bk[i] = H->bk[i];
        }
    }
    const double2 g2 = __ldg(P.grow + k);
    const int first = u - c;
    Acc t{0.0, 0, -1};
    for (int i = lane; i < npc; i += 32) {
        t.minfin = __dadd_rn(t.minfin, __ldcg(A.hpart + first + i));
        const int2 pi = __ldcg(A.hpinf + first + i);
        t.ninf += pi.x;
        t.infj = max(t.infj, pi.y);
    }
    t = warp_reduce(t);
    const bool infeasible = row_infeasible(t.minfin, t.ninf, g2.y);
    if (c == 0 && lane == 0) {
        atomicAdd(&st.nnz, (unsigned long long)(re - beg));
        atomicAdd(&st.i_nnz[ki], (unsigned long long)(re - beg));
        if (infeasible) atomicMin(&A.i_rowinf[ph.s3() * A.ninst + ki], k);
    }
    if (infeasible || t.ninf >= 2) return;
    if (!H) load_elems(E, P, ph, beg, end, lane, 32);
    elems_candidates(st, A, P, ph, E, t, g2.x);
}

__device__ void do_fix(const Stage& st, const BpArgs& A, const DevProblem& P, const Phase& ph, const int* chg_prev,
                       int nprev, int tl);

// Warp task tl of phase A after the pieces: [fix-ups][thread-per-row bins][warp rows].
__device__ __forceinline__ void warp_task(Stage& st, const BpArgs& A, const DevProblem& P, const Phase& ph, int tl,
                                          const int* rows, const int* cnt, const int* s_bin, int s_fix,
                                          const int* chg_prev, int nprev) {
    if (tl < s_fix) {
        do_fix(st, A, P, ph, chg_prev, nprev, tl);
        return;
    }
    tl -= s_fix;
#pragma unroll
    for (int c = 0; c < kNumThreadBins; ++c) {
        if (tl < s_bin[c]) {
            do_thread_rows(st, A, P, ph, rows + P.class_off[c], cnt[c], tl);
            return;
        }
        tl -= s_bin[c];
    }
    do_warp_row(st, A, P, ph, __ldcg(rows + P.class_off[kClassWarpRow] + tl));
}

// Variables changed in the previous round: bring their new bounds into this round's
// write buffer (atomic, so it commutes with this round's tightenings) and check crossings.
__device__ void do_fix(const Stage& st, const BpArgs& A, const DevProblem& P, const Phase& ph, const int* chg_prev,
                       int nprev, int tl) {
    const int idx = tl * 32 + (threadIdx.x & 31);
    if (idx >= nprev) return;
    const int v = __ldcg(chg_prev + idx);
    const int vi = var_inst(st, A, v);
    if (!st.alive[vi] && !st.pending[vi]) return;
    const longlong2 b = ld_bounds(ph.R, v);
    if (st.alive[vi]) {
        atomicMax(&ph.X[v].x, b.x);
        atomicMin(&ph.X[v].y, b.y);
    }
    if (crossed(P.is_int[v] != 0, b.x, b.y)) atomicMin(&A.i_cross[ph.s3() * A.ninst + vi], v);
}

// -------------------------------------------------------------------- barrier
// Grid barrier: every block arrives once on a count that only grows within the launch and
// waits until all blocks have arrived at this barrier (the launch's bar_k-th).  No block
// resets anything or releases the others, so no bookkeeping sits on the others' path: after
// the barrier each block reads the round's counters itself and takes the same decisions.
// The arrival is one acquire-release atomic of thread 0 after the block barrier (release is
// cumulative over the writes the block barrier ordered before it) and the wait a tight spin of
// acquire loads: on GB300 a separate fence costs 450-950 cycles and a sleep in the spin at least
// 500 cycles of reaction time, and both sit on every round's critical path.
__device__ void grid_sync(Stage& st, Ctl* ctl) {
    __syncthreads();
    if (threadIdx.x == 0) {
        atom_add_acqrel_u32(&ctl->bar_count.v, 1u);
        const unsigned target = gridDim.x * (st.bar_k + 1u);
        const long long t0 = clock64();
        while (ld_acquire_u32(&ctl->bar_count.v) < target) {
            if (clock64() - t0 > kSpinLimit) {
                atomicExch(&ctl->error, BP_ERR_TIMEOUT);
                break;
            }
        }
        st.bar_k += 1u;
    }
    __syncthreads();
}

// Descriptor of round `next` into shared memory (thread 0): its worklist counts per class,
// its pieces and the previous round's changed variables.
__device__ __forceinline__ void load_descriptor(Stage& st, Ctl* ctl, const DevProblem& P, const BpArgs& A,
                                                int next) {
    const int sl = next % kPhaseSlots;
    const bool stat = (next == 0 && !A.w0 && !A.w0v);
#pragma unroll
    for (int c = 0; c < kNumClass; ++c)
        st.d_cnt[c] = stat ? P.class_off[c + 1] - P.class_off[c] : __ldcg(&ctl->cnt[sl][c].v);
    st.d_ntask = stat ? P.npieces : __ldcg(&ctl->ntask[sl].v);
    st.d_nprev = next == 0 ? 0 : __ldcg(&ctl->nchg[(next - 1) % kPhaseSlots].v);
}

// After the barrier that ends round t.  Every block takes the instances' verdicts of round t
// from the same counters, so all reach the same live / pending flags and result buffers (kept
// in shared memory), reads the descriptor of round t+1 and decides whether to stop.  Block 0
// also records the verdicts in the instance states, writes the trace, and clears the counter
// slots that round t+2 appends to: slot t % 3 of the worklist counts and slot (t+2) % 3 of the
// rest, whose last readers finished before this barrier.
__device__ __noinline__ void end_round(Stage& st, Ctl* ctl, const DevProblem& P, const BpArgs& A, int t) {
    const int sl = t % kPhaseSlots, sl1 = (t + 1) % kPhaseSlots, sl2 = (t + 2) % kPhaseSlots;
    const int par = t & 1, npar = par ^ 1;
    const bool writer = blockIdx.x == 0;
    // thread 0: the descriptor of round t+1, the error flag and the round's nonzeros, loaded
    // together with the verdict words below (one round trip)
    int d_cnt[kNumClass], d_ntask = 0, d_nprev = 0, err = 0, rows_t = 0;
    unsigned long long nnz_t = 0;
    if (threadIdx.x == 0) {
#pragma unroll
        for (int c = 0; c < kNumClass; ++c) {
            rows_t += st.d_cnt[c];
            d_cnt[c] = __ldcg(&ctl->cnt[sl1][c].v);
        }
        d_ntask = __ldcg(&ctl->ntask[sl1].v);
        d_nprev = __ldcg(&ctl->nchg[sl].v);
        err = __ldcg(&ctl->error);
        if (writer && A.trace) nnz_t = __ldcg(&ctl->nnz[sl].v);
    }
    int any_alive = 0;
    for (int i = threadIdx.x; i < A.ninst; i += kThreads) {
        const int cross = __ldcg(A.i_cross + sl * A.ninst + i);
        const int rinf = __ldcg(A.i_rowinf + sl * A.ninst + i);
        const int chg = __ldcg(A.i_chg + sl * A.ninst + i);
        int alive = st.alive[i], pending = st.pending[i];
        if (alive) {
            InstState* I = A.inst + i;
            if (cross != INT_MAX) {
                // bounds after round t-1 cross: that round is the instance's last
                alive = 0;
                st.rpar[i] = (unsigned char)par;
                if (writer) {
                    I->status = BP_INFEASIBLE;
                    I->rounds = t;
                    I->result_par = par;
                    I->first_var = cross;
                    I->first_row = INT_MAX;
                }
            } else {
                st.rpar[i] = (unsigned char)npar;
                int status = -1;
                if (rinf != INT_MAX) {
                    status = BP_INFEASIBLE;
                    alive = 0;
                    pending = 1;     // crossing check of this round's changes
                } else if (!chg) {
                    status = BP_FIXPOINT;
                    alive = 0;
                } else if (t + 1 >= A.max_rounds) {
                    status = BP_ROUND_LIMIT;
                    alive = 0;
                    pending = 1;
                }
                if (writer) {
                    I->nnz_total = __ldcg(&I->nnz_total) + __ldcg(A.i_nnz + sl * A.ninst + i);
                    I->rounds = t + 1;
                    I->result_par = npar;
                    if (status >= 0) I->status = status;
                    if (rinf != INT_MAX) I->first_row = rinf;
                    I->pending = pending;
                }
            }
            if (writer) I->alive = alive;
        } else if (pending) {
            // the crossing check of the instance's last round ran in this round
            pending = 0;
            if (writer) {
                InstState* I = A.inst + i;
                if (cross != INT_MAX && cross < __ldcg(&I->first_var)) I->first_var = cross;
                I->pending = 0;
            }
        }
        st.alive[i] = (unsigned char)alive;
        st.pending[i] = (unsigned char)pending;
        st.i_nnz[i] = 0;
        any_alive |= alive;
        if (writer) {
            A.i_nnz[sl2 * A.ninst + i] = 0;
            A.i_rowinf[sl2 * A.ninst + i] = INT_MAX;
            A.i_cross[sl2 * A.ninst + i] = INT_MAX;
            A.i_chg[sl2 * A.ninst + i] = 0;
        }
    }
    any_alive = __syncthreads_or(any_alive);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int c = 0; c < kNumClass; ++c) st.d_cnt[c] = d_cnt[c];
        st.d_ntask = d_ntask;
        st.d_nprev = d_nprev;
        st.flag = (!any_alive || err) ? 1 : 0;
        st.epi_n = d_nprev;   // variables changed in round t (checked at the end when it is the last)
        st.epi_par = par;
        if (writer) {
            if (A.trace && t < A.max_rounds) {
                A.trace[4 * t + 0] = rows_t;
                A.trace[4 * t + 1] = (long long)nnz_t;
                A.trace[4 * t + 2] = d_nprev;
                A.trace[4 * t + 3] = (long long)globaltimer_ns();
            }
            ctl->phases = t + 1;
#pragma unroll
            for (int c = 0; c < kNumClass; ++c) ctl->cnt[sl][c].v = 0;
            ctl->ntask[sl].v = 0;
            ctl->nchg[sl2].v = 0;
            ctl->nnz[sl2].v = 0;
        }
    }
    __syncthreads();
}

// Flushes the block's per-instance nonzero counts of round slot `sl`.
__device__ void flush_inst_nnz(Stage& st, const BpArgs& A, int sl) {
    __syncthreads();
    for (int i = threadIdx.x; i < A.ninst; i += kThreads)
        if (st.i_nnz[i]) atomicAdd(&A.i_nnz[sl * A.ninst + i], st.i_nnz[i]);
    __syncthreads();
}

__device__ void finish_block(Stage& st, const BpArgs& A) {
    // the last block out writes the result slots
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        st.last_block = atom_add_acqrel_u32(&A.ctl->done.v, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!st.last_block) return;
    __threadfence();
    const int err = __ldcg(&A.ctl->error);
    if (threadIdx.x == 0) {
        const int b0 = __ldcg(A.stamp);
        const int b = b0 > (1 << 30) ? 1 : b0;
        *A.stamp = b + __ldcg(&A.ctl->phases) + 3;
    }
    for (int i = threadIdx.x; i < A.ninst; i += kThreads) {
        const InstState* I = A.inst + i;
        bp_result r;
        r.error = err;
        r.status = __ldcg(&I->status);
        r.rounds = __ldcg(&I->rounds);
        const int fr = __ldcg(&I->first_row), fv = __ldcg(&I->first_var);
        r.first_infeasible_row = fr == INT_MAX ? -1 : fr;
        r.first_infeasible_var = fv == INT_MAX ? -1 : fv;
        if (r.first_infeasible_var >= 0) r.status = BP_INFEASIBLE;
        r.nnz_updates = (int64_t)__ldcg(&I->nnz_total);
        r.n_changed = (int64_t)__ldcg(&I->n_changed);
        r.reserved = 0;
        A.dres[i] = r;
    }
}

// The Jacobi rounds of one propagation, from the round-0 descriptor in `st` until every
// instance has stopped (or the error flag is set).  Stamps of round t: base + t.
__device__ __forceinline__ void run_rounds(Stage& st, const DevProblem& P, const BpArgs& A, int base) {
    Ctl* ctl = A.ctl;
    const int gw_r = (threadIdx.x >> 5) * gridDim.x + blockIdx.x;
    const int NW = gridDim.x * kWarpsPerBlock;
    for (int t = 0; !st.flag; ++t) {
        Phase ph;
        ph.t = t;
        ph.par = t & 1;
        ph.npar = ph.par ^ 1;
        ph.R = A.bk[ph.par];
        ph.X = A.bk[ph.npar];
        ph.st_v = base + t;
        ph.st_r = base + t + 1;
        const bool stat = (t == 0 && !A.w0 && !A.w0v);
        const int* rows = stat ? P.static_list : A.list[ph.par];
        const int4* tasks = stat ? P.static_tasks : A.task[ph.par];
        const int ntask = st.d_ntask;
        const int nprev = st.d_nprev;
        const int* chg_prev = A.chg[ph.npar];
        int cnt[kNumClass];
#pragma unroll
        for (int c = 0; c < kNumClass; ++c) cnt[c] = st.d_cnt[c];
        // phase A, warp tasks: pieces of piece rows (partials), fix-ups of the previous round's
        // changes, thread-per-row bins, warp rows
        const int s_fix = (nprev + 31) / 32;
        int s_bin[kNumThreadBins];
        int total = ntask + s_fix + cnt[kClassWarpRow];
#pragma unroll
        for (int c = 0; c < kNumThreadBins; ++c) {
            s_bin[c] = (cnt[c] + 31) / 32;
            total += s_bin[c];
        }
        // with at most one task per warp (short rounds), a piece's warp keeps its nonzeros and
        // bounds in registers from phase A to phase B
        const bool single = total <= NW;
        HeldBounds H1;
        int4 tk1 = make_int4(0, 0, 0, 0);
        bool piece1 = false;
        if (single) {
            if (gw_r < ntask) {
                tk1 = __ldcg(tasks + gw_r);
                piece1 = st.alive[row_inst(st, A, tk1.x)] != 0;
                if (piece1) piece_partial(A, P, ph, gw_r, tk1, &H1);
            } else if (gw_r < total) {
                warp_task(st, A, P, ph, gw_r - ntask, rows, cnt, s_bin, s_fix, chg_prev, nprev);
            }
        } else {
            for (int task = gw_r; task < total; task += NW) {
                if (task < ntask) {
                    const int4 tk = __ldcg(tasks + task);
                    if (st.alive[row_inst(st, A, tk.x)]) piece_partial(A, P, ph, task, tk, nullptr);
                } else {
                    warp_task(st, A, P, ph, task - ntask, rows, cnt, s_bin, s_fix, chg_prev, nprev);
                }
            }
        }
        // phase B: every piece's row total and candidates, once all partials are written
        if (ntask > 0) {
            grid_sync(st, ctl);
            if (single) {
                if (piece1) piece_candidates(st, A, P, ph, gw_r, tk1, &H1);
            } else {
                for (int task = gw_r; task < ntask; task += NW) {
                    const int4 tk = __ldcg(tasks + task);
                    if (st.alive[row_inst(st, A, tk.x)]) piece_candidates(st, A, P, ph, task, tk, nullptr);
                }
            }
        }
        // changes of this block: dedupe grid-wide, list them, queue their rows
        drain_changed(st, A, P, ph);
        // staged appends to the global lists; nonzeros of this phase: one atomic per block
        warp_flush_all(st, A, P, ph);
        __syncthreads();
        if (threadIdx.x == 0 && st.nnz) {
            atomicAdd(&ctl->nnz[ph.s3()].v, st.nnz);
            st.nnz = 0;
        }
        flush_inst_nnz(st, A, ph.s3());
        if (A.skip_block == (int)blockIdx.x) {
            // test-only failure: this block stops arriving at the grid barrier, so the others'
            // bounded waits run out and the launch reports BP_ERR_TIMEOUT
            st.flag = 2;
            break;
        }
        grid_sync(st, ctl);
        end_round(st, ctl, P, A, t);
    }

}

// After the round-0 lists are queued (and a grid barrier): every block decides which instances
// run round 0 (block 0 records the others' verdicts) and loads the round-0 descriptor.
__device__ __forceinline__ void round0_state(Stage& st, const DevProblem& P, const BpArgs& A) {
    Ctl* ctl = A.ctl;
    int rows0 = 0;
    if (A.w0 || A.w0v)
        for (int c = 0; c < kNumClass; ++c) rows0 += __ldcg(&ctl->cnt[0][c].v);
    if (threadIdx.x == 0) st.any_alive = 0;
    __syncthreads();
    for (int i = threadIdx.x; i < A.ninst; i += kThreads) {
        InstState* I = A.inst + i;
        // rows in round 0: with a variable start list and several instances, each
        // instance's own (a nonzero count is all that matters here)
        const int ri = (A.w0v && A.ninst > 1) ? __ldcg(&I->start_rows)
                       : (A.w0 || A.w0v)      ? rows0
                                              : st.roff[i + 1] - st.roff[i];
        const int ec = __ldcg(&I->entry_cross);
        int alive = 1;
        if (ec != INT_MAX) {
            alive = 0;
            if (blockIdx.x == 0) {
                I->status = BP_INFEASIBLE;
                I->first_var = ec;
            }
        } else if (ri == 0 || A.max_rounds <= 0) {
            alive = 0;
            if (blockIdx.x == 0) I->status = ri == 0 ? BP_FIXPOINT : BP_ROUND_LIMIT;
        }
        if (blockIdx.x == 0) I->alive = alive;
        st.alive[i] = (unsigned char)alive;
        if (alive) atomicOr(&st.any_alive, 1);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        load_descriptor(st, ctl, P, A, 0);
        st.flag = (!st.any_alive || __ldcg(&ctl->error)) ? 1 : 0;
    }
    __syncthreads();
}

// Crossing check of the last round of the instances whose check is pending (their last
// round's changed variables).
__device__ __forceinline__ void last_round_cross(Stage& st, const DevProblem& P, const BpArgs& A) {
    const int gtid = blockIdx.x * blockDim.x + threadIdx.x, gthreads = gridDim.x * blockDim.x;
    const int epi_n = st.epi_n;
    if (epi_n > 0) {
        // crossing check of the last round of the instances whose check is pending
        const int* lst = A.chg[st.epi_par];
        for (int i = gtid; i < epi_n; i += gthreads) {
            const int v = __ldcg(lst + i);
            const int vi = var_inst(st, A, v);
            if (!st.pending[vi]) continue;
            const longlong2 b = __ldcg(A.bk[st.rpar[vi]] + v);
            if (crossed(P.is_int[v] != 0, b.x, b.y)) atomicMin(&A.inst[vi].first_var, v);
        }
    }
}

// ---------------------------------------------------------------------- kernel
__global__ void __launch_bounds__(kThreads, GPUBP_MIN_BLOCKS) bp_kernel(DevProblem P, BpArgs A) {
    __shared__ Stage st;
    const int lane = threadIdx.x & 31;
    // warp tasks are numbered across blocks first, so that a short round's few tasks land on
    // different SMs
    const int gw_r = (threadIdx.x >> 5) * gridDim.x + blockIdx.x;
    const int NW = gridDim.x * kWarpsPerBlock;
    const int gtid = blockIdx.x * blockDim.x + threadIdx.x, gthreads = gridDim.x * blockDim.x;
    Ctl* ctl = A.ctl;
    for (int i = threadIdx.x; i < kWarpsPerBlock * kSlots; i += kThreads) (&st.wcnt[0][0])[i] = 0;
    if (threadIdx.x == 0) {
        st.bq_n = 0;
        st.nnz = 0;
        st.bar_k = 0;
        st.epi_n = 0;
        st.epi_par = 0;
    }
    for (int i = threadIdx.x; i < A.ninst; i += kThreads) {
        st.alive[i] = 1;
        st.pending[i] = 0;
        st.rpar[i] = 0;
        st.i_nnz[i] = 0;
    }
    for (int i = threadIdx.x; i <= A.ninst; i += kThreads) {
        st.roff[i] = A.ninst == 1 ? (i ? P.m : 0) : A.row_off[i];
        st.coff[i] = A.ninst == 1 ? (i ? P.n : 0) : A.col_off[i];
    }
    // stamps: this launch's round t uses base + t; the base lives on the device so that a
    // replayed CUDA graph keeps advancing it; when it grows large the stamp arrays restart
    int base = __ldcg(A.stamp);
    if (base > (1 << 30)) {
        for (int v = gtid; v < P.n; v += gthreads) A.vstamp[v] = 0;
        for (int k = gtid; k < P.m; k += gthreads) A.rstamp[k] = 0;
        base = 1;
    }
    // per-instance state and per-phase arrays
    for (int i = gtid; i < A.ninst; i += gthreads) {
        InstState I;
        I.status = BP_FIXPOINT;
        I.rounds = 0;
        I.result_par = 0;
        I.first_row = INT_MAX;
        I.first_var = INT_MAX;
        I.alive = 1;
        I.pending = 0;
        I.entry_cross = INT_MAX;
        I.start_rows = 0;
        I.nnz_total = 0;
        I.n_changed = 0;
        A.inst[i] = I;
        for (int q = 0; q < kPhaseSlots; ++q) {
            A.i_nnz[q * A.ninst + i] = 0;
            A.i_rowinf[q * A.ninst + i] = INT_MAX;
            A.i_cross[q * A.ninst + i] = INT_MAX;
            A.i_chg[q * A.ninst + i] = 0;
        }
    }
    __syncthreads();
    // all instance state must be initialised before any block updates it
    grid_sync(st, ctl);

    // ---- prologue: normalised start bounds into both buffers; rows of round 0
    for (int v = gtid; v < P.n; v += gthreads) {
        const bool is_i = P.is_int[v] != 0;
        const longlong2 b = normalized_keys(A.lb[v], A.ub[v], is_i);
        A.bk[0][v] = b;
        A.bk[1][v] = b;
        if (crossed(is_i, b.x, b.y)) atomicMin(&A.inst[var_inst(st, A, v)].entry_cross, v);
    }
    Phase ph0{0, 0, 1, A.bk[0], A.bk[1], base, base};
    if (A.w0) {
        // queue the given rows into the round-0 lists (stamp `base` = member of round 0)
        Phase q = ph0;
        q.npar = 0;     // round 0's list and counter slot (t = -1: next slot 0)
        q.t = -1;
        const int gw0 = gtid >> 5, nw0 = gthreads >> 5;
        for (int b = gw0 * 32; b < A.w0_len; b += nw0 * 32) {
            const int i = b + lane;
            warp_queue_rows(st, A, P, q, i < A.w0_len ? __ldg(A.w0 + i) : -1);
        }
        warp_flush_all(st, A, P, q);
    } else if (A.w0v) {
        // queue the rows of the given variables (one warp per variable)
        Phase q = ph0;
        q.npar = 0;     // round 0's list and counter slot (t = -1: next slot 0)
        q.t = -1;
        const int gw0 = gtid >> 5, nw0 = gthreads >> 5;
        const int nv = *A.w0v_len;
        for (int b = gw0; b < nv; b += nw0) {
            const int u = __ldg(A.w0v + b);
            if (u < 0 || u >= P.n) {   // caller's index out of range: skipped, reported
                if (lane == 0) atomicExch(&ctl->error, BP_ERR_INVALID);
                continue;
            }
            const int cb = __ldg(P.col_ptr + u), ce = __ldg(P.col_ptr + u + 1);
            if (A.ninst > 1 && lane == 0 && ce > cb) atomicAdd(&A.inst[var_inst(st, A, u)].start_rows, 1);
            for (int s0 = cb; s0 < ce; s0 += 32) {
                const int sidx = s0 + lane;
                warp_queue_rows(st, A, P, q, sidx < ce ? __ldg(P.row_idx + sidx) : -1);
            }
        }
        warp_flush_all(st, A, P, q);
    }
    grid_sync(st, ctl);
    // every block: which instances run round 0
    round0_state(st, P, A);

    // ---- rounds
    run_rounds(st, P, A, base);

    // ---- epilogue
    if (st.flag != 2 && !ld_acquire_s32(&ctl->error)) {
        last_round_cross(st, P, A);
        for (int vb = blockIdx.x * kThreads; vb < P.n; vb += gthreads) {
            const int v = vb + threadIdx.x;
            int changed = 0, vi = -1;
            if (v < P.n) {
                vi = var_inst(st, A, v);
                const longlong2 in = normalized_keys(A.lb[v], A.ub[v], P.is_int[v] != 0);
                const longlong2 b = __ldcg(A.bk[st.rpar[vi]] + v);
                changed = (b.x != in.x || b.y != in.y) ? 1 : 0;
                A.lb[v] = kdec(b.x);
                A.ub[v] = kdec(b.y);
            }
            // one atomic per instance present in the warp
            const unsigned peers = __match_any_sync(0xffffffffu, vi);
            const int total = __popc(__ballot_sync(0xffffffffu, changed) & peers);
            if (vi >= 0 && lane == __ffs(peers) - 1 && total) atomicAdd(&A.inst[vi].n_changed, (unsigned long long)total);
        }
    }
    finish_block(st, A);
}

// ------------------------------------------------- device-driven single fixings (Section 2.3)
// fix_and_propagate's one-variable bulks (the recovery of a failed bulk, Algorithm 1) run in one
// persistent launch over the instance pair: for each queued variable still unfixed, the two
// candidate values (the draw and the other rounding) are fixed in the two copies, both copies
// propagate from that variable's rows (the same rounds as run_rounds in a launch of their own),
// and the first feasible candidate becomes the current bounds.  The current bounds stay ordered
// keys on the device between fixings; only the variables a propagation changed (the dirty list)
// are copied back into the pair's buffers, so a fixing costs its rounds, not a pass over n.
struct FpSingleArgs {
    longlong2* cur;            // n0: the current bounds (ordered keys)
    const int* queue;          // variables to fix one at a time, in order
    int qlen;
    int n0;                    // variables of one copy
    const double* x;
    const double* up_prob;
    unsigned long long seed, bulk0;
    int* words;                // [0..1] start list, [2] its length, [3] dirty count
    FpSingleOut* out;
    unsigned char* chosen;     // or NULL: kept fixings are recorded (the repair's fixings by choice)
    double* cval;
};

__global__ void __launch_bounds__(kThreads, GPUBP_MIN_BLOCKS) fp_single_kernel(DevProblem P, BpArgs A, FpSingleArgs F) {
    __shared__ Stage st;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int gtid = blockIdx.x * blockDim.x + threadIdx.x, gthreads = gridDim.x * blockDim.x;
    Ctl* ctl = A.ctl;
    const int n0 = F.n0;
    for (int i = threadIdx.x; i < kWarpsPerBlock * kSlots; i += kThreads) (&st.wcnt[0][0])[i] = 0;
    if (threadIdx.x == 0) {
        st.bq_n = 0;
        st.nnz = 0;
        st.bar_k = 0;
    }
    for (int i = threadIdx.x; i <= A.ninst; i += kThreads) {
        st.roff[i] = A.row_off[i];
        st.coff[i] = A.col_off[i];
    }
    int base = __ldcg(A.stamp);
    long long bulks = 0, runs = 0, nnz = 0, fixed = 0;
    int infeasible = 0, stop_q = -1, stop_j = -1;
    __shared__ double s_val[2];   // block 0: the current variable's two candidate values
    __syncthreads();
    for (int q = 0; q < F.qlen; ++q) {
        if (base > (1 << 30)) {
            // the stamps restart (every block sees the same base)
            for (int v = gtid; v < P.n; v += gthreads) {
                A.vstamp[v] = 0;
                A.vdirty[v] = 0;
            }
            for (int k = gtid; k < P.m; k += gthreads) A.rstamp[k] = 0;
            base = 1;
            grid_sync(st, ctl);
        }
        const int j = __ldg(F.queue + q);
        if (threadIdx.x == 0) {
            int go = 0;
            if ((unsigned)j < (unsigned)n0) {
                const longlong2 c = __ldcg(F.cur + j);
                go = c.x < c.y ? 1 : 0;     // fixed meanwhile: skipped, no bulk
            } else if (gtid == 0) {
                atomicExch(&ctl->error, BP_ERR_INVALID);
            }
            st.go = go;
        }
        __syncthreads();
        const int go = st.go;
        __syncthreads();
        if (!go) continue;
        // this propagation's block state
        for (int i = threadIdx.x; i < A.ninst; i += kThreads) {
            st.alive[i] = 1;
            st.pending[i] = 0;
            st.rpar[i] = 0;
            st.i_nnz[i] = 0;
        }
        if (threadIdx.x == 0) {
            st.epi_n = 0;
            st.epi_par = 0;
            st.dstamp = base;
        }
        if (blockIdx.x == 0) {
            // block 0: counters, instance states, the two candidate fixings (the draw in copy 0,
            // the other rounding in copy 1), the start list and the rows of round 0
            if (threadIdx.x == 0) {
                for (int q3 = 0; q3 < kPhaseSlots; ++q3) {
#pragma unroll
                    for (int c = 0; c < kNumClass; ++c) ctl->cnt[q3][c].v = 0;
                    ctl->ntask[q3].v = 0;
                    ctl->nchg[q3].v = 0;
                    ctl->nnz[q3].v = 0;
                }
                ctl->phases = 0;
                for (int i = 0; i < A.ninst; ++i) {
                    InstState I;
                    I.status = BP_FIXPOINT;
                    I.rounds = 0;
                    I.result_par = 0;
                    I.first_row = INT_MAX;
                    I.first_var = INT_MAX;
                    I.alive = 1;
                    I.pending = 0;
                    I.entry_cross = INT_MAX;
                    I.start_rows = 0;
                    I.nnz_total = 0;
                    I.n_changed = 0;
                    A.inst[i] = I;
                    for (int q3 = 0; q3 < kPhaseSlots; ++q3) {
                        A.i_nnz[q3 * A.ninst + i] = 0;
                        A.i_rowinf[q3 * A.ninst + i] = INT_MAX;
                        A.i_cross[q3 * A.ninst + i] = INT_MAX;
                        A.i_chg[q3 * A.ninst + i] = 0;
                    }
                }
                const longlong2 c = __ldcg(F.cur + j);
                const double l = kdec(c.x), u = kdec(c.y);
                const double xh = clampd(__ldg(F.x + j), l, u);
                const double va = clampd(draw_value(xh, F.seed, F.bulk0 + (unsigned long long)bulks, j, 0, F.up_prob), l, u);
                const double fl = floor(xh);
                const double vb = clampd(va == fl ? __dadd_rn(fl, 1.0) : fl, l, u);
                const bool is_i = P.is_int[j] != 0;
                const longlong2 ka = normalized_keys(va, va, is_i), kb = normalized_keys(vb, vb, is_i);
                s_val[0] = va;
                s_val[1] = vb;
                A.bk[0][j] = ka;
                A.bk[1][j] = ka;
                A.bk[0][n0 + j] = kb;
                A.bk[1][n0 + j] = kb;
                if (crossed(is_i, ka.x, ka.y)) A.inst[0].entry_cross = j;
                if (crossed(is_i, kb.x, kb.y)) A.inst[1].entry_cross = n0 + j;
                A.vdirty[j] = base;
                A.vdirty[n0 + j] = base;
                A.dirty[0] = j;
                A.dirty[1] = n0 + j;
                *A.ndirty = 2;
                F.words[0] = j;
                F.words[1] = n0 + j;
                F.words[2] = 2;
                __threadfence();
            }
            __syncthreads();
            Phase qph{0, 0, 1, A.bk[0], A.bk[1], base, base};
            qph.npar = 0;     // round 0's list and counter slot (t = -1: next slot 0)
            qph.t = -1;
            if (warp < 2) {
                const int u = warp == 0 ? j : n0 + j;
                const int cb = __ldg(P.col_ptr + u), ce = __ldg(P.col_ptr + u + 1);
                if (lane == 0 && ce > cb) atomicAdd(&A.inst[warp].start_rows, 1);
                for (int s0 = cb; s0 < ce; s0 += 32) {
                    const int sidx = s0 + lane;
                    warp_queue_rows(st, A, P, qph, sidx < ce ? __ldg(P.row_idx + sidx) : -1);
                }
            }
            warp_flush_all(st, A, P, qph);
        }
        grid_sync(st, ctl);
        round0_state(st, P, A);
        run_rounds(st, P, A, base);
        if (ld_acquire_s32(&ctl->error)) break;
        last_round_cross(st, P, A);
        grid_sync(st, ctl);
        // every block reads the same verdicts and picks the same candidate
        if (threadIdx.x == 0) {
            int pick = -1;
            for (int c = 1; c >= 0; --c) {
                const int status = __ldcg(&A.inst[c].status), fv = __ldcg(&A.inst[c].first_var);
                if (status != BP_INFEASIBLE && fv == INT_MAX) pick = c;
            }
            st.go = pick;
        }
        __syncthreads();
        const int pick = st.go;
        // the changed variables of both copies back to the current bounds (the picked copy's
        // values when a candidate is feasible)
        const int nd = __ldcg(A.ndirty);
        const longlong2* R = pick >= 0 ? A.bk[st.rpar[pick]] : nullptr;
        for (int i = gtid; i < nd; i += gthreads) {
            const int d = __ldcg(A.dirty + i);
            const int b = d < n0 ? d : d - n0;
            longlong2 kv;
            if (pick >= 0) {
                kv = __ldcg(R + (size_t)pick * n0 + b);
                F.cur[b] = kv;
            } else {
                kv = __ldcg(F.cur + b);
            }
            A.bk[0][b] = kv;
            A.bk[1][b] = kv;
            A.bk[0][n0 + b] = kv;
            A.bk[1][n0 + b] = kv;
        }
        if (gtid == 0) {
            bulks += 1;
            runs += 2;
            nnz += (long long)(__ldcg(&A.inst[0].nnz_total) + __ldcg(&A.inst[1].nnz_total));
            if (pick >= 0) {
                fixed += 1;
                if (F.chosen) {
                    F.chosen[j] = 1;
                    F.cval[j] = s_val[pick];
                }
            } else {
                infeasible = 1;
                stop_q = q;
                stop_j = j;
                F.out->v0 = s_val[0];
            }
        }
        base += __ldcg(&ctl->phases) + 3;
        grid_sync(st, ctl);
        if (pick < 0) break;
    }
    if (gtid == 0) {
        const int err = __ldcg(&ctl->error);
        F.out->bulks = bulks;
        F.out->bp_runs = runs;
        F.out->nnz_updates = nnz;
        F.out->fixed = fixed;
        F.out->infeasible = infeasible;
        F.out->error = err;
        F.out->stop_q = stop_q;
        F.out->j = stop_j;
        // a propagation cut short by an error may have used stamps up to base + max_rounds + 1
        *A.stamp = err ? base + A.max_rounds + 3 : base;
    }
}

// ------------------------------------------------------------------------ host
void ctl_template(Ctl* c) { memset(c, 0, sizeof(Ctl)); }

static int ensure_instances(mip_problem* p, int ninst) {
    Work& w = p->w;
    if (ninst <= w.inst_cap) return BP_OK;
    BP_TRY(dalloc(p, &w.dres, (size_t)ninst));
    BP_TRY(dalloc(p, &w.inst, (size_t)ninst));
    BP_TRY(dalloc(p, &w.i_nnz, kPhaseSlots * (size_t)ninst));
    BP_TRY(dalloc(p, &w.i_rowinf, kPhaseSlots * (size_t)ninst));
    BP_TRY(dalloc(p, &w.i_cross, kPhaseSlots * (size_t)ninst));
    BP_TRY(dalloc(p, &w.i_chg, kPhaseSlots * (size_t)ninst));
    w.inst_cap = ninst;
    return BP_OK;
}

int engine_prepare(mip_problem* p) {
    Work& w = p->w;
    const int m = p->m, n = p->n;
    BP_TRY(dalloc(p, &w.bkey[0], (size_t)n));
    BP_TRY(dalloc(p, &w.bkey[1], (size_t)n));
    BP_TRY(dalloc(p, &w.vstamp, (size_t)n));
    BP_TRY(dalloc(p, &w.rstamp, (size_t)m));
    BP_TRY(dalloc(p, &w.list[0], (size_t)m));
    BP_TRY(dalloc(p, &w.list[1], (size_t)m));
    BP_TRY(dalloc(p, &w.chg[0], (size_t)n));
    BP_TRY(dalloc(p, &w.chg[1], (size_t)n));
    BP_TRY(dalloc(p, &w.task[0], (size_t)p->chunk_cap));
    BP_TRY(dalloc(p, &w.task[1], (size_t)p->chunk_cap));
    BP_TRY(dalloc(p, &w.hpart, (size_t)p->chunk_cap));
    BP_TRY(dalloc(p, &w.hpinf, (size_t)p->chunk_cap));
    BP_TRY(dalloc(p, &w.ctl, 1));
    BP_TRY(ensure_instances(p, 1));
    BP_TRY(dalloc(p, &w.stage_lb, (size_t)n));
    BP_TRY(dalloc(p, &w.stage_ub, (size_t)n));
    void* h = nullptr;
    BP_CUDA_TRY(cudaMallocHost(&h, sizeof(Ctl)));
    p->host_allocs.push_back(h);
    w.ctl_host = static_cast<Ctl*>(h);
    ctl_template(w.ctl_host);
    {
        const int one = 1;
        BP_TRY(dalloc(p, &w.stamp, 1));
        BP_CUDA_TRY(cudaMemcpy(w.stamp, &one, sizeof(int), cudaMemcpyHostToDevice));
    }
    // persistent grid: every block must be resident (cooperative launch)
    int occ = 0;
    BP_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, bp_kernel, kThreads, 0));
    int sms = 0;
    BP_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->device));
    if (occ < 1) {
        set_error("propagation kernel cannot be resident on this device");
        return BP_ERR_CUDA;
    }
    p->sms = sms;
    p->occ_max = occ > 4 ? 4 : occ;
    p->grid_blocks = sms * p->occ_max;
    // the no-allocation entry point's static scratch is reserved here, with the handle's other
    // memory, never by that entry point's first call
    BP_TRY(noalloc_prepare(p->device));
    return BP_OK;
}

int launch_propagate(mip_problem* p, double* lb, double* ub, const int* w0, int w0_len, double theta,
                     int max_rounds, int64_t* trace, cudaStream_t s, const int* w0v, const int* w0v_len, int ninst,
                     const int* row_off, const int* col_off) {
    Work& w = p->w;
    if (ninst < 1 || ninst > kMaxInstances || (ninst > 1 && (!row_off || !col_off || w0))) {
        set_error("invalid instance batch (1 <= instances <= %d, offsets required, no row start list)",
                  kMaxInstances);
        return BP_ERR_INVALID;
    }
    BP_TRY(ensure_instances(p, ninst));
    BpArgs a;
    a.lb = lb;
    a.ub = ub;
    a.bk[0] = w.bkey[0];
    a.bk[1] = w.bkey[1];
    a.vstamp = w.vstamp;
    a.rstamp = w.rstamp;
    a.list[0] = w.list[0];
    a.list[1] = w.list[1];
    a.chg[0] = w.chg[0];
    a.chg[1] = w.chg[1];
    a.task[0] = w.task[0];
    a.task[1] = w.task[1];
    a.hpart = w.hpart;
    a.hpinf = w.hpinf;
    a.ctl = w.ctl;
    a.dres = w.dres;
    a.w0 = w0;
    a.w0_len = w0_len;
    a.w0v = w0v;
    a.w0v_len = w0v_len;
    a.theta = theta;
    a.max_rounds = max_rounds;
    a.stamp = w.stamp;
    a.trace = (long long*)trace;
    // test-only failure injection: GPUBP_TEST_SKIP_BLOCK=b makes block b leave the rounds
    // without arriving at the grid barrier (the failure-detection tests; never set otherwise)
    {
        const char* e = getenv("GPUBP_TEST_SKIP_BLOCK");
        a.skip_block = (e && *e) ? atoi(e) : -1;
    }
    a.ninst = ninst;
    a.row_off = row_off;
    a.col_off = col_off;
    a.inst = w.inst;
    a.i_nnz = w.i_nnz;
    a.i_rowinf = w.i_rowinf;
    a.i_cross = w.i_cross;
    a.i_chg = w.i_chg;
    a.vdirty = nullptr;
    a.dirty = nullptr;
    a.ndirty = nullptr;
    BP_CUDA_TRY(cudaMemcpyAsync(w.ctl, w.ctl_host, sizeof(Ctl), cudaMemcpyHostToDevice, s));
    DevProblem dp = p->dp;
    void* args[] = {&dp, &a};
    BP_CUDA_TRY(cudaLaunchCooperativeKernel((const void*)bp_kernel, dim3(p->grid_blocks), dim3(kThreads), args, 0, s));
    p->last_stream = s;
    return BP_OK;
}

int launch_fp_single(mip_problem* tw, int n0, longlong2* cur, const int* queue, int qlen, const double* x,
                     const double* up_prob, unsigned long long seed, unsigned long long bulk0, double theta,
                     int max_rounds, int* vdirty, int* dirty, int* words, FpSingleOut* out, unsigned char* chosen,
                     double* cval, cudaStream_t s) {
    Work& w = tw->w;
    if (!tw->inst_row_off || !tw->inst_col_off || 2 * (long long)n0 != tw->n) {
        set_error("launch_fp_single: not an instance pair");
        return BP_ERR_INVALID;
    }
    BP_TRY(ensure_instances(tw, 2));
    static int occ_single = -1;
    if (occ_single < 0) {
        int occ = 0;
        BP_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fp_single_kernel, kThreads, 0));
        occ_single = occ;
    }
    if (occ_single < 1) {
        set_error("fix-and-propagate kernel cannot be resident on this device");
        return BP_ERR_CUDA;
    }
    const int occ = occ_single < tw->occ_max ? occ_single : tw->occ_max;
    BpArgs a;
    a.lb = nullptr;
    a.ub = nullptr;
    a.bk[0] = w.bkey[0];
    a.bk[1] = w.bkey[1];
    a.vstamp = w.vstamp;
    a.rstamp = w.rstamp;
    a.list[0] = w.list[0];
    a.list[1] = w.list[1];
    a.chg[0] = w.chg[0];
    a.chg[1] = w.chg[1];
    a.task[0] = w.task[0];
    a.task[1] = w.task[1];
    a.hpart = w.hpart;
    a.hpinf = w.hpinf;
    a.ctl = w.ctl;
    a.dres = w.dres;
    a.w0 = nullptr;
    a.w0_len = 0;
    a.w0v = words;
    a.w0v_len = words + 2;
    a.theta = theta;
    a.max_rounds = max_rounds;
    a.stamp = w.stamp;
    a.trace = nullptr;
    a.skip_block = -1;
    a.ninst = 2;
    a.row_off = tw->inst_row_off;
    a.col_off = tw->inst_col_off;
    a.inst = w.inst;
    a.i_nnz = w.i_nnz;
    a.i_rowinf = w.i_rowinf;
    a.i_cross = w.i_cross;
    a.i_chg = w.i_chg;
    a.vdirty = vdirty;
    a.dirty = dirty;
    a.ndirty = words + 3;
    FpSingleArgs f;
    f.cur = cur;
    f.queue = queue;
    f.qlen = qlen;
    f.n0 = n0;
    f.x = x;
    f.up_prob = up_prob;
    f.seed = seed;
    f.bulk0 = bulk0;
    f.words = words;
    f.out = out;
    f.chosen = chosen;
    f.cval = cval;
    BP_CUDA_TRY(cudaMemcpyAsync(w.ctl, w.ctl_host, sizeof(Ctl), cudaMemcpyHostToDevice, s));
    DevProblem dp = tw->dp;
    void* args[] = {&dp, &a, &f};
    BP_CUDA_TRY(cudaLaunchCooperativeKernel((const void*)fp_single_kernel, dim3(tw->sms * occ), dim3(kThreads), args, 0, s));
    tw->last_stream = s;
    return BP_OK;
}

}  // namespace gpubp

using namespace gpubp;

extern "C" int bp_propagate(mip_problem* p, double* lb, double* ub, const bp_params* params, bp_result* result,
                            void* stream) {
    if (!p || (p->n && (!lb || !ub))) {
        set_error("null argument");
        return BP_ERR_INVALID;
    }
    bp_params prm;
    if (params) {
        prm = *params;
    } else {
        bp_params_default(&prm);
    }
    if (!(prm.theta >= 0.0) || prm.max_rounds < 0 ||
        (prm.bounds_mem != BP_MEM_DEVICE && prm.bounds_mem != BP_MEM_HOST)) {
        set_error("invalid parameters (theta >= 0, max_rounds >= 0, bounds_mem host/device)");
        return BP_ERR_INVALID;
    }
    cudaStream_t s = (cudaStream_t)stream;
    double *dl = lb, *du = ub;
    const size_t bytes = sizeof(double) * (size_t)p->n;
    if (prm.bounds_mem == BP_MEM_HOST) {
        dl = p->w.stage_lb;
        du = p->w.stage_ub;
        if (p->n) {
            BP_CUDA_TRY(cudaMemcpyAsync(dl, lb, bytes, cudaMemcpyHostToDevice, s));
            BP_CUDA_TRY(cudaMemcpyAsync(du, ub, bytes, cudaMemcpyHostToDevice, s));
        }
    }
    BP_TRY(launch_propagate(p, dl, du, nullptr, 0, prm.theta, prm.max_rounds, prm.trace, s));
    if (prm.bounds_mem == BP_MEM_HOST && p->n) {
        BP_CUDA_TRY(cudaMemcpyAsync(lb, dl, bytes, cudaMemcpyDeviceToHost, s));
        BP_CUDA_TRY(cudaMemcpyAsync(ub, du, bytes, cudaMemcpyDeviceToHost, s));
    }
    if (result) BP_CUDA_TRY(cudaMemcpyAsync(result, p->w.dres, sizeof(bp_result), cudaMemcpyDeviceToHost, s));
    return BP_OK;
}

extern "C" const bp_result* bp_result_device(const mip_problem* p) { return p ? p->w.dres : nullptr; }

extern "C" int bp_propagate_from(mip_problem* p, double* lb, double* ub, const int32_t* vars, int32_t nvars,
                                 const bp_params* params, bp_result* result, void* stream) {
    if (!p || nvars < 0 || (nvars && !vars) || (p->n && (!lb || !ub))) {
        set_error("bp_propagate_from: null or negative argument");
        return BP_ERR_INVALID;
    }
    bp_params prm;
    if (params) prm = *params;
    else bp_params_default(&prm);
    if (!(prm.theta >= 0.0) || prm.max_rounds < 0 || prm.bounds_mem != BP_MEM_DEVICE) {
        set_error("bp_propagate_from: invalid parameters (device bounds only)");
        return BP_ERR_INVALID;
    }
    cudaStream_t s = (cudaStream_t)stream;
    Work& w = p->w;
    if (!w.nvars_dev) BP_TRY(dalloc(p, &w.nvars_dev, 1));
    BP_CUDA_TRY(cudaMemcpyAsync(w.nvars_dev, &nvars, sizeof(int), cudaMemcpyHostToDevice, s));
    BP_TRY(launch_propagate(p, lb, ub, nullptr, 0, prm.theta, prm.max_rounds, prm.trace, s, vars ? vars : w.nvars_dev,
                            w.nvars_dev));
    if (result) BP_CUDA_TRY(cudaMemcpyAsync(result, p->w.dres, sizeof(bp_result), cudaMemcpyDeviceToHost, s));
    return BP_OK;
}
