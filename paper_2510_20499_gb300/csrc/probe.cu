// Batched double probing (Section 2.2): bp_probe_batch.
//
// A probe propagation starts from the rows of one variable and usually stays small, so a grid
// barrier per round would cost more than the work.  Each thread block therefore runs whole
// probe pairs on its own: it takes a pair (both branches of one variable) from a counter and
// runs their Jacobi rounds with block barriers only.  The two branches are propagated
// together ("double propagation", Section 2.2): a worklist row carries a mask of the branches
// whose worklist holds it, and one load of its coefficients and columns serves both.
//
// Bounds of a branch are root ∩ scratch, where the block's dense scratch holds neutral keys
// (-inf, +inf) except for the variables the branch tightened; only those are reset after a
// pair, so neither the root nor the scratch is ever copied in full.  Stamps are 64-bit epochs
// that only grow, so no stamp array is ever cleared.
#include <climits>

#include "bp_host.h"

namespace gpubp {

#ifndef GPUBP_PROBE_THREADS
#define GPUBP_PROBE_THREADS 128
#endif
#ifndef GPUBP_PROBE_BLOCKS_PER_SM
#define GPUBP_PROBE_BLOCKS_PER_SM 6
#endif
#ifndef GPUBP_PROBE_GLANES
#define GPUBP_PROBE_GLANES 0                   // lanes per worklist row; 0 = chosen from the row lengths
#endif
constexpr int kPThreads = GPUBP_PROBE_THREADS;     // a pair's few rows per round need few warps
constexpr int kPBlocksPerSM = GPUBP_PROBE_BLOCKS_PER_SM;
constexpr size_t kPScratchBudget = (size_t)16 << 30;   // bytes of per-block scratch at most
constexpr size_t kPDenseBudget = (size_t)1 << 30;      // bytes of the dense pass's per-variable scratch
constexpr int kPWarps = kPThreads / 32;
constexpr int kPLane = 4;                  // nonzeros per lane held in registers per segment
constexpr int kPSort = 4096;               // touched lists up to this size are sorted in shared memory
constexpr int kHCapMax = 2048;             // slots per block in the sparse pass
constexpr long long kPSpinLimit = 4000000000LL;   // clock64 cycles (about 2 s) of a bounded wait

struct ProbeArgs {
    const longlong2* root;       // n root keys
    const float* rowcap;         // m: per-row cap of the candidate filter at the root (k_probe_rowcap)
    const int* var;
    const double* boxes;         // 4 per pair
    int npairs;
    // per-variable state lives in `cap` slots: in the sparse pass a slot of the block's hash
    // table of the variables the pair touched (table in shared memory, cap = kHCap, scratch
    // strided by block); in the dense pass the variable itself (cap = n, scratch strided by
    // dense slot)
    longlong2* S;                // [2 branch][2 parity][cap]
    unsigned long long* vst;     // [2 branch][cap]  last epoch a variable changed
    unsigned long long* rw;      // [m]  (epoch << 2) | branch mask of the row's worklist entry
    int* wl;                     // [2 parity][m]
    int* chg;                    // [2 branch][2 parity][cap]  slots
    int* touched;                // [2 branch][cap]  slots
    unsigned long long* ep;      // [1] epoch counter of the block
    int* pair_ctr;
    int* ovf;                    // [npairs] pairs the sparse pass left to the dense pass (-1: none)
    int* novf;                   // their count
    int* ovf_ctr;                // next overflow pair of the dense pass
    int* done;                   // blocks that finished the sparse pass
    int dense_blocks;            // dense scratch slots
    longlong2* Sd;               // dense scratch, per slot as S, vst, chg, touched with cap = n
    unsigned long long* vstd;
    int* chgd;
    int* touchedd;
    unsigned long long* epd;     // [dense_blocks] epoch counter of each dense slot
    int glanes;                  // lanes per worklist row: 8, 16 or 32 (a warp takes 32 / glanes rows)
    double theta;
    int max_rounds;
    // outputs
    int* status;
    int* rounds;
    int64_t* nnzu;
    long long* ecount;           // per branch: entries
    long long* estart;           // per branch: start in the temp arrays
    int64_t* offsets;            // [2 npairs + 1] the cache's entry offsets (written by the last block)
    int* evar;
    double* el;
    double* eu;
    unsigned long long* ectr;
    long long ecap;
    int* error;
};

__device__ __forceinline__ longlong2 neutral_keys() { return make_longlong2(kKeyNegInf, kKeyPosInf); }

__device__ __forceinline__ longlong2 meet(longlong2 r, longlong2 s) {
    return make_longlong2(r.x > s.x ? r.x : s.x, r.y < s.y ? r.y : s.y);
}

__device__ __forceinline__ long long box_key(double x) {
    if (x <= -kInfBound) return kKeyNegInf;
    if (x >= kInfBound) return kKeyPosInf;
    return dkey(x);
}

struct ProbeShared {
    int pair, v;
    int alive[2];
    int status[2], rounds[2];
    unsigned long long nnz[2];
    int rowinf[2], cross[2];
    int nw[2];                   // worklist entries per parity
    int wcount[2][2];            // [parity][branch] entries holding the branch
    int nchg[2][2];              // [branch][parity]
    int ntouch[2];
    unsigned long long ep_pair, ep_t, ep;
    int hkey[kHCapMax];          // the slot table, variable + 1 (0 = free)
    int hfull;                   // the pair touched more variables than the table holds
    int last;                    // this block finished the sparse pass last
    union {
        int sortbuf[kPSort];     // output phase: the touched variables being sorted
        struct {                 // rows phase: each warp's queue of candidates that passed the filter
            double a[kPWarps][32], mf[kPWarps][32], g[kPWarps][32];
            long long lk[kPWarps][32], uk[kPWarps][32];
            int j[kPWarps][32], bn[kPWarps][32];   // variable; branch | (infinite terms << 1)
        } q;
    };
    int scan[kPThreads];
    int out_base;
};

// Per-variable slots and the pair's touched variables.  The block's shared-memory table holds
// the variables the pair touched (open addressing with linear probing on a multiplicative
// hash's high bits; all entries are freed after the pair, so a chain never crosses a free
// entry, and a variable inserted during the current round still has neutral current-round
// bounds, so a lookup that misses it reads the right values).  A variable outside the table has
// its root bounds in both branches, so its gathers read the (L2-resident) root keys and skip
// the scratch.  Sparse pass: a variable's slot is its table entry, and a pair that does not
// fit is left to the dense pass.  Dense pass: the slot is the variable itself and the table
// only filters; once full it answers "touched" for every variable, which only costs the
// scratch read.
constexpr int kHCap = kHCapMax;
constexpr int kHProbe = 64;      // probes before the table counts as full for the pair
static_assert(kHCap <= kPSort && (kHCap & (kHCap - 1)) == 0, "table size");

__device__ __forceinline__ unsigned hslot(int j) { return __umulhi((unsigned)j * 2654435761u, (unsigned)kHCap); }

// the slot of a touched variable, -1 for one the pair has not touched
__device__ __forceinline__ int slot_find(const ProbeShared& sh, bool dense, int j) {
    if (dense && sh.hfull) return j;
    const volatile int* hk = sh.hkey;
    unsigned h = hslot(j);
    for (int q = 0; q < kHProbe; ++q) {
        const int k = hk[h];
        if (k == j + 1) return dense ? j : (int)h;
        if (k == 0) return -1;
        h = (h + 1) & (unsigned)(kHCap - 1);
    }
    return dense ? j : -1;
}

// the slot of j, entered in the table if new; when the table is full the pair is marked
// (sparse pass: -1, the pair goes to the dense pass)
__device__ __forceinline__ int slot_get(ProbeShared& sh, bool dense, int j) {
    volatile int* hk = sh.hkey;
    unsigned h = hslot(j);
    for (int q = 0; q < kHProbe; ++q) {
        int k = hk[h];
        if (k == j + 1) return dense ? j : (int)h;
        if (k == 0) {
            k = atomicCAS(&sh.hkey[h], 0, j + 1);
            if (k == 0 || k == j + 1) return dense ? j : (int)h;
        }
        h = (h + 1) & (unsigned)(kHCap - 1);
    }
    sh.hfull = 1;
    return dense ? j : -1;
}

__device__ __forceinline__ int slot_var(const ProbeShared& sh, bool dense, int sl) {
    return dense ? sl : reinterpret_cast<const volatile int*>(sh.hkey)[sl] - 1;
}

__device__ __forceinline__ bool positive(double a) { return __double_as_longlong(a) >= 0; }   // a != 0

// Per-row cap of the candidate filter for a probe batch.  A branch's bounds lie inside the root
// bounds, so for every nonzero the filter's product |a| (u - l) is at most its value at the root
// and its margin term 2e-15 |a| (|l'| + |u'|) at most 4e-15 |a| (|l| + |u|) (|l'| + |u'| <=
// 2 max(|l|, |u|) for l <= l' <= u' <= u).  The cap is the maximum over the row of the product
// plus twice that bound (FP32, rounded up; +inf when a bound is infinite); the factor two, and
// 2e-15 in place of 1e-15 on |g| + |L_min| below, absorb the different order of the upward
// roundings.  A row whose slack bracket reaches cap + 2e-15 (|g| + |L_min|) lets no candidate
// through the per-nonzero filter in any branch, so the filter loop is skipped.
__global__ void k_probe_rowcap(DevProblem P, const longlong2* root, float* cap, int* pair_ctr,
                               unsigned long long* ectr, int G) {
    const int lane = threadIdx.x & 31, gl = lane & (G - 1);
    if (blockIdx.x == 0 && threadIdx.x == 0) {   // the launch's counters: next pair, entry total, index flag
        pair_ctr[0] = 0;
        pair_ctr[1] = 0;
        pair_ctr[2] = 0;
        pair_ctr[3] = 0;
        ectr[0] = 0;
        ectr[1] = 0;
    }
    // a group of G lanes per row, 32 / G rows per warp at a time (warp-uniform loop: the
    // reduction's shuffles are warp-wide)
    const int rpw = 32 / G;
    const int wi = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int kb = wi * rpw; kb < P.m; kb += nwarps * rpw) {
        const int k = kb + lane / G;
        const bool live = k < P.m;
        float c = 0.0f;
        if (live) {
            for (int q = P.row_ptr[k] + gl; q < P.row_ptr[k + 1]; q += G) {
                const longlong2 b = root[P.col[q]];
                if (key_is_inf(b.x) || key_is_inf(b.y)) {
                    c = __int_as_float(0x7f800000);
                    continue;
                }
                const double l = kdec(b.x), u = kdec(b.y);
                const float a_up = fabs_up(P.val[q]);
                const float prod = __fmul_ru(a_up, __fsub_ru(f_up(u), f_dn(l)));
                const float mt = __fmul_ru(1e-15f, __fmul_ru(8.0f, __fmul_ru(a_up, __fadd_ru(fabs_up(l), fabs_up(u)))));
                c = fmaxf(c, __fadd_ru(prod, mt));
            }
        }
        for (int off = G >> 1; off > 0; off >>= 1) c = fmaxf(c, __shfl_xor_sync(0xffffffffu, c, off));
        if (live && gl == 0) cap[k] = c;
    }
}

// Per-variable scratch of one pair: `cap` slots (see ProbeArgs).
struct PairScratch {
    int cap;
    longlong2* S;
    unsigned long long* vst;
    int* chg;
    int* touched;
};

// Both branches of one pair, by one block.  Sparse pass (dense = false): per-variable state in
// the block's compact scratch at the variable's table entry; a pair that fills the table is
// freed and listed for the dense pass.  Dense pass: slot = variable.
__device__ __forceinline__ void probe_pair(ProbeShared& sh, const DevProblem& P, const ProbeArgs& A,
                                           const PairScratch& sc, unsigned long long* rw, int* wl, int pair,
                                           bool dense) {
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int n = P.n, m = P.m;
    const int cap = sc.cap;
    longlong2* S = sc.S;
    unsigned long long* vst = sc.vst;
    int* chg = sc.chg;
    int* touched = sc.touched;
    auto Sb = [&](int b, int p) { return S + (size_t)(2 * b + p) * cap; };
    auto chgb = [&](int b, int p) { return chg + (size_t)(2 * b + p) * cap; };
    const unsigned long long ep_pair = sh.ep_pair;
    if (dense) {
        // the table only filters in the dense pass: cleared per pair
        for (int i = tid; i < kHCap; i += kPThreads) sh.hkey[i] = 0;
        __syncthreads();
    }
    // ---- branch set-up: start box = root ∩ branch box of the probed variable
    if (tid < 2) {
        const int b = tid;
        const int v = A.var[pair];
        if (v < 0 || v >= n) {   // caller's index out of range: the call reports BP_ERR_INVALID
            if (b == 0) atomicExch(A.error, 1);
            sh.v = -1;
        } else {
        const longlong2 r = A.root[v];
        const longlong2 bx = make_longlong2(box_key(A.boxes[4 * pair + 2 * b]), box_key(A.boxes[4 * pair + 2 * b + 1]));
        const longlong2 s0 = meet(r, bx);
        const int sv = slot_get(sh, dense, v);   // an empty table: always found
        Sb(b, 0)[sv] = s0;
        Sb(b, 1)[sv] = s0;
        vst[(size_t)b * cap + sv] = ep_pair;
        touched[(size_t)b * cap] = sv;
        sh.ntouch[b] = 1;
        sh.nnz[b] = 0;
        sh.rounds[b] = 0;
        sh.v = v;
        if (crossed(P.is_int[v] != 0, s0.x, s0.y)) {
            sh.status[b] = BP_INFEASIBLE;
            sh.alive[b] = 0;
        } else {
            sh.status[b] = BP_FIXPOINT;
            sh.alive[b] = 1;
        }
        sh.nchg[b][0] = sh.nchg[b][1] = 0;
        sh.wcount[0][b] = 0;
        }
    }
    if (tid == 0) sh.nw[0] = 0;
    __syncthreads();
    if (sh.v < 0) return;
    // ---- round 0 worklist: the rows of the probed variable, for the live branches
    const int v = sh.v;
    const unsigned mask0 = (unsigned)(sh.alive[0] | (sh.alive[1] << 1));
    if (mask0) {
        const int cb = P.col_ptr[v], ce = P.col_ptr[v + 1];
        for (int s = cb + tid; s < ce; s += kPThreads) {
            const int k = P.row_idx[s];
            rw[k] = (ep_pair << 2) | mask0;
            wl[s - cb] = k;
        }
        if (tid == 0) {
            sh.nw[0] = ce - cb;
            sh.wcount[0][0] = (mask0 & 1) ? ce - cb : 0;
            sh.wcount[0][1] = (mask0 & 2) ? ce - cb : 0;
        }
    }
    __syncthreads();

    for (int t = 0;; ++t) {
        const int par = t & 1, np = par ^ 1;
        // branches whose worklist is empty or that hit the round limit stop here
        if (tid < 2) {
            const int b = tid;
            if (sh.alive[b]) {
                if (sh.wcount[par][b] == 0) {
                    sh.alive[b] = 0;
                    sh.status[b] = BP_FIXPOINT;
                    sh.rounds[b] = t;
                } else if (t >= A.max_rounds) {
                    sh.alive[b] = 0;
                    sh.status[b] = BP_ROUND_LIMIT;
                    sh.rounds[b] = t;
                }
            }
            sh.rowinf[b] = 0;
            sh.cross[b] = 0;
            sh.nchg[b][par] = 0;
            sh.wcount[np][b] = 0;
        }
        if (tid == 0) {
            sh.nw[np] = 0;
            sh.ep_t = ++sh.ep;
        }
        __syncthreads();
        const unsigned live = (unsigned)(sh.alive[0] | (sh.alive[1] << 1));
        if (!live || (!dense && sh.hfull)) break;
        const unsigned long long ep_t = sh.ep_t;
        // fix-ups of the previous round's changes into this round's write buffers
        if (t > 0) {
            for (int b = 0; b < 2; ++b) {
                if (!(live >> b & 1)) continue;
                const int nprev = sh.nchg[b][np];
                const int* cl = chgb(b, np);
                longlong2* R = Sb(b, par);
                longlong2* X = Sb(b, np);
                for (int i = tid; i < nprev; i += kPThreads) {
                    const int u = cl[i];
                    const longlong2 rv = R[u];
                    atomicMax(&X[u].x, rv.x);
                    atomicMin(&X[u].y, rv.y);
                }
            }
        }
        // ---- rows of this round: a group of G lanes per row (32 / G rows per warp at a
        // time, so that the short rows of a probe overlap their load latencies), both branches
        // per load
        const int nw = sh.nw[par];
        const int* W = wl + (size_t)par * m;
        const int G = A.glanes, gpw = 32 / G, gl = lane & (G - 1);
        const int seg = G * kPLane;
        for (int e0 = w * gpw; e0 < nw; e0 += kPWarps * gpw) {
            const int e = e0 + lane / G;
            const int k = e < nw ? W[e] : -1;
            const unsigned mask = k >= 0 ? (unsigned)(rw[k] & 3ull) & live : 0u;
            if (!__any_sync(0xffffffffu, mask != 0)) continue;
            int beg = 0, end = 0;
            double2 g2 = make_double2(0.0, 0.0);
            float rcap = 0.0f;
            if (mask) {
                beg = P.row_ptr[k];
                end = P.row_ptr[k + 1];
                g2 = P.grow[k];
                rcap = A.rowcap[k];
            }
            double mf[2] = {0.0, 0.0};
            int ni[2] = {0, 0}, ij[2] = {-1, -1};
            int jj[kPLane];
            double aa[kPLane];
            long long kk[2][kPLane];   // per branch: the bound key of the minimum contribution
            for (int s0 = beg; s0 < end; s0 += seg) {
#pragma unroll
                for (int i = 0; i < kPLane; ++i) {
                    const int q = s0 + gl + G * i;
                    jj[i] = q < end ? P.col[q] : -1;
                    aa[i] = q < end ? P.val[q] : 0.0;
                }
#pragma unroll
                for (int i = 0; i < kPLane; ++i) {
                    if (jj[i] < 0) continue;
                    // only the bound of the minimum contribution: l for a > 0, u for a < 0
                    const bool pos = positive(aa[i]);
                    const int sj = slot_find(sh, dense, jj[i]);
                    const long long r = __ldcg(reinterpret_cast<const long long*>(A.root) + 2 * jj[i] + (pos ? 0 : 1));
#pragma unroll
                    for (int b = 0; b < 2; ++b) {
                        long long x = r;
                        if ((mask >> b & 1) && sj >= 0) {
                            const long long y =
                                __ldcg(reinterpret_cast<const long long*>(Sb(b, par)) + 2 * sj + (pos ? 0 : 1));
                            x = pos ? (y > r ? y : r) : (y < r ? y : r);
                        }
                        kk[b][i] = x;
                    }
                }
#pragma unroll
                for (int i = 0; i < kPLane; ++i) {
                    if (jj[i] < 0) continue;
#pragma unroll
                    for (int b = 0; b < 2; ++b) {
                        if (!(mask >> b & 1)) continue;
                        const long long key = kk[b][i];
                        if (key_is_inf(key)) {
                            ++ni[b];
                            ij[b] = jj[i];
                        } else {
                            mf[b] = fma(aa[i], kdec(key), mf[b]);
                        }
                    }
                }
            }
            // group reductions (xor offsets below G stay inside the group)
#pragma unroll
            for (int b = 0; b < 2; ++b) {
                for (int off = G >> 1; off > 0; off >>= 1) {
                    mf[b] = __dadd_rn(mf[b], __shfl_xor_sync(0xffffffffu, mf[b], off));
                    ni[b] += __shfl_xor_sync(0xffffffffu, ni[b], off);
                    ij[b] = max(ij[b], __shfl_xor_sync(0xffffffffu, ij[b], off));
                }
            }
            // Candidates: the FP32 filter runs per nonzero; the few that pass go to the warp's
            // queue, and the exact FP64 evaluation (a division, slow on this part) runs once per
            // 32 queued candidates with every lane busy, instead of once per register slot that
            // has a candidate in some lane.
            int qn = 0;   // warp-uniform queue length
            auto flush = [&]() {
                __syncwarp();
                if (lane < qn) {
                    const int j = sh.q.j[w][lane], bn = sh.q.bn[w][lane], b = bn & 1;
                    const long long lk = sh.q.lk[w][lane], uk = sh.q.uk[w][lane];
                    long long nk;
                    const int r = eval_candidate(sh.q.a[w][lane], lk, uk, sh.q.mf[w][lane], bn >> 1, sh.q.g[w][lane],
                                                 P.is_int[j] != 0, A.theta, &nk);
                    const int sj = r ? slot_get(sh, dense, j) : -1;
                    if (sj >= 0) {
                        longlong2* X = Sb(b, np);
                        if (r == 1) atomicMin(&X[sj].y, nk);
                        else atomicMax(&X[sj].x, nk);
                        const unsigned long long old = atomicMax(&vst[(size_t)b * cap + sj], ep_t);
                        if (old < ep_t) chgb(b, par)[atomicAdd(&sh.nchg[b][par], 1)] = sj;
                        if (old < ep_pair) touched[(size_t)b * cap + atomicAdd(&sh.ntouch[b], 1)] = sj;
                    }
                }
                __syncwarp();
                qn = 0;
            };
#pragma unroll
            for (int b = 0; b < 2; ++b) {
                bool rowok = false;
                RowFilter f{};
                if (mask >> b & 1) {
                    if (gl == 0) atomicAdd(&sh.nnz[b], (unsigned long long)(end - beg));
                    if (row_infeasible(mf[b], ni[b], g2.y)) {
                        if (gl == 0) sh.rowinf[b] = 1;
                    } else if (ni[b] < 2) {
                        f = row_filter(g2.x, mf[b]);
                        // the row-level cap (NaN-safe: an infinite cap keeps the filter loop)
                        rowok = !(ni[b] == 0 && f.slack_dn >= __fadd_ru(rcap, __fmul_ru(2e-15f, f.mag_up)));
                    }
                }
                if (!__any_sync(0xffffffffu, rowok)) continue;
                const int nseg = rowok ? (end - beg + seg - 1) / seg : 0;
                const int nseg_w = __reduce_max_sync(0xffffffffu, nseg);
                for (int si = 0; si < nseg_w; ++si) {
                    const int s0 = beg + si * seg;
#pragma unroll
                    for (int i = 0; i < kPLane; ++i) {
                        bool want = false;
                        int j = -1;
                        double a = 0.0;
                        longlong2 bk = make_longlong2(0, 0);
                        // the row's nonzeros are read again (L2) rather than held in registers
                        // since the activity pass: few rows get here, and the freed registers
                        // let more blocks share an SM
                        const int q = s0 + gl + G * i;
                        if (si < nseg && q < end) {
                            j = P.col[q];
                            a = P.val[q];
                            const int sj = slot_find(sh, dense, j);
                            bk = sj >= 0 ? meet(__ldcg(A.root + j), __ldcg(Sb(b, par) + sj)) : __ldcg(A.root + j);
                            want = ni[b] == 1 ? j == ij[b] : !cannot_tighten(f, a, bk.x, bk.y);
                        }
                        const unsigned bal = __ballot_sync(0xffffffffu, want);
                        if (bal) {
                            if (qn + __popc(bal) > 32) flush();
                            if (want) {
                                unsigned lt;
                                asm("mov.u32 %0, %%lanemask_lt;" : "=r"(lt));
                                const int pos = qn + __popc(bal & lt);
                                sh.q.a[w][pos] = a;
                                sh.q.mf[w][pos] = mf[b];
                                sh.q.g[w][pos] = g2.x;
                                sh.q.lk[w][pos] = bk.x;
                                sh.q.uk[w][pos] = bk.y;
                                sh.q.j[w][pos] = j;
                                sh.q.bn[w][pos] = b | (ni[b] << 1);
                            }
                            qn += __popc(bal);
                        }
                    }
                }
            }
            if (qn) flush();
        }
        __syncthreads();
        // ---- verdicts of the round: infeasible rows, crossing bounds
        for (int b = 0; b < 2; ++b) {
            if (!(live >> b & 1) || sh.rowinf[b]) continue;
            const int nc = sh.nchg[b][par];
            const int* cl = chgb(b, par);
            const longlong2* X = Sb(b, np);
            for (int i = tid; i < nc; i += kPThreads) {
                const int sl = cl[i], u = slot_var(sh, dense, sl);
                const longlong2 x = meet(__ldcg(A.root + u), __ldcg(X + sl));
                if (crossed(P.is_int[u] != 0, x.x, x.y)) sh.cross[b] = 1;
            }
        }
        __syncthreads();
        if (tid < 2) {
            const int b = tid;
            if (live >> b & 1) {
                sh.rounds[b] = t + 1;
                if (sh.rowinf[b] || sh.cross[b]) {
                    sh.alive[b] = 0;
                    sh.status[b] = BP_INFEASIBLE;
                }
            }
        }
        __syncthreads();
        // ---- next worklist: rows of the variables changed in this round
        for (int b = 0; b < 2; ++b) {
            if (!sh.alive[b]) continue;
            const int nc = sh.nchg[b][par];
            const int* cl = chgb(b, par);
            const unsigned bit = 1u << b;
            // warp per changed variable, lanes over its rows
            for (int i = w; i < nc; i += kPWarps) {
                const int u = slot_var(sh, dense, cl[i]);
                const int cb = P.col_ptr[u], ce = P.col_ptr[u + 1];
                for (int s = cb + lane; s < ce; s += 32) {
                    const int k = P.row_idx[s];
                    unsigned long long old = rw[k], nv;
                    bool first;
                    do {
                        first = (old >> 2) != ep_t;
                        if (!first && (old & bit)) break;
                        nv = first ? ((ep_t << 2) | bit) : (old | bit);
                        const unsigned long long seen = atomicCAS(&rw[k], old, nv);
                        if (seen == old) {
                            atomicAdd(&sh.wcount[np][b], 1);
                            if (first) wl[(size_t)np * m + atomicAdd(&sh.nw[np], 1)] = k;
                            break;
                        }
                        old = seen;
                    } while (true);
                }
            }
        }
        __syncthreads();
    }

    if (!dense && sh.hfull) {
        // the table could not hold the pair's variables: its slots are freed and the pair
        // goes to the dense pass, which writes all of its outputs
        for (int b = 0; b < 2; ++b) {
            const int* tl = touched + (size_t)b * cap;
            for (int i = tid; i < sh.ntouch[b]; i += kPThreads) {
                const int u = tl[i];
                Sb(b, 0)[u] = neutral_keys();
                Sb(b, 1)[u] = neutral_keys();
            }
        }
        __syncthreads();
        for (int b = 0; b < 2; ++b)
            for (int i = tid; i < sh.ntouch[b]; i += kPThreads) sh.hkey[touched[(size_t)b * cap + i]] = 0;
        if (tid == 0) A.ovf[atomicAdd(A.novf, 1)] = pair;
        __syncthreads();
        return;
    }
    // ---- outputs of the pair
    for (int b = 0; b < 2; ++b) {
        const int e = 2 * pair + b;
        const bool feas = sh.status[b] != BP_INFEASIBLE;
        const int nt = sh.ntouch[b];
        const int* tl = touched + (size_t)b * cap;
        const longlong2* F = Sb(b, sh.rounds[b] & 1);
        if (!feas || nt <= 32) {
            // few touched variables (the usual case): one warp sorts them with shuffles and
            // writes the entries that differ from the root, in variable order
            if (w == 0) {
                // (variable, slot) packed, sorted by variable
                long long xs = LLONG_MAX;
                if (feas && lane < nt) {
                    const int sl = tl[lane];
                    xs = ((long long)slot_var(sh, dense, sl) << 32) | (unsigned)sl;
                }
                for (int k = 2; k <= 32; k <<= 1) {
                    for (int j = k >> 1; j > 0; j >>= 1) {
                        const long long y = __shfl_xor_sync(0xffffffffu, xs, j);
                        xs = (((lane & j) == 0) == ((lane & k) == 0)) ? min(xs, y) : max(xs, y);
                    }
                }
                const int x = xs == LLONG_MAX ? INT_MAX : (int)(xs >> 32);
                int d = 0;
                longlong2 xv = make_longlong2(0, 0);
                if (x != INT_MAX) {
                    const longlong2 r = A.root[x];
                    xv = meet(r, __ldcg(F + (int)(xs & 0xffffffffll)));
                    d = (xv.x != r.x || xv.y != r.y) ? 1 : 0;
                }
                const unsigned msk = __ballot_sync(0xffffffffu, d);
                const int cnt = __popc(msk);
                unsigned long long base = 0;
                if (lane == 0) {
                    A.status[e] = sh.status[b];
                    A.rounds[e] = sh.rounds[b];
                    A.nnzu[e] = (int64_t)sh.nnz[b];
                    A.ecount[e] = cnt;
                    base = cnt ? atomicAdd(A.ectr, (unsigned long long)cnt) : 0ull;
                    A.estart[e] = (long long)base;
                }
                base = __shfl_sync(0xffffffffu, base, 0);
                if (d) {
                    unsigned lt;
                    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(lt));
                    const long long pos = (long long)base + __popc(msk & lt);
                    if (pos < A.ecap) {
                        A.evar[pos] = x;
                        A.el[pos] = kdec(xv.x);
                        A.eu[pos] = kdec(xv.y);
                    }
                }
            }
            __syncthreads();
        } else {
        // sorted touched variables: in shared memory (the next power of two at or above the
        // count) when few, else in index order from the stamps
        const bool small = !dense || nt <= kPSort;   // the sparse pass holds at most kHCap <= kPSort
        if (small) {
            int p2 = 64;
            while (p2 < nt) p2 <<= 1;
            for (int i = tid; i < p2; i += kPThreads) sh.sortbuf[i] = i < nt ? slot_var(sh, dense, tl[i]) : INT_MAX;
            __syncthreads();
            for (int size = 2; size <= p2; size <<= 1) {
                for (int stride = size >> 1; stride > 0; stride >>= 1) {
                    for (int i = tid; i < p2; i += kPThreads) {
                        const int jx = i ^ stride;
                        if (jx > i) {
                            const bool up = (i & size) == 0;
                            const int x = sh.sortbuf[i], y = sh.sortbuf[jx];
                            if ((x > y) == up) {
                                sh.sortbuf[i] = y;
                                sh.sortbuf[jx] = x;
                            }
                        }
                    }
                    __syncthreads();
                }
            }
        }
        // count the entries that differ from the root, in variable order
        const int span = small ? nt : n;
        long long cnt = 0;
        for (int base = 0; base < span; base += kPThreads) {
            const int i = base + tid;
            int u = -1;
            if (i < span) u = small ? sh.sortbuf[i] : (vst[(size_t)b * cap + i] >= ep_pair ? i : -1);
            int d = 0;
            if (u >= 0) {
                const longlong2 r = A.root[u];
                const longlong2 x = meet(r, __ldcg(F + (dense ? u : slot_find(sh, false, u))));
                d = (x.x != r.x || x.y != r.y) ? 1 : 0;
            }
            sh.scan[tid] = d;
            __syncthreads();
            for (int o = 1; o < kPThreads; o <<= 1) {
                const int y = tid >= o ? sh.scan[tid - o] : 0;
                __syncthreads();
                sh.scan[tid] += y;
                __syncthreads();
            }
            cnt += sh.scan[kPThreads - 1];
            __syncthreads();
        }
        if (tid == 0) {
            sh.out_base = (int)0;
            A.status[e] = sh.status[b];
            A.rounds[e] = sh.rounds[b];
            A.nnzu[e] = (int64_t)sh.nnz[b];
            A.ecount[e] = cnt;
            const unsigned long long base = cnt ? atomicAdd(A.ectr, (unsigned long long)cnt) : 0ull;
            A.estart[e] = (long long)base;
            sh.ep_t = base;   // reuse as the write base
        }
        __syncthreads();
        const unsigned long long wbase = sh.ep_t;
        long long written = 0;
        for (int base = 0; base < span && cnt; base += kPThreads) {
            const int i = base + tid;
            int u = -1;
            if (i < span) u = small ? sh.sortbuf[i] : (vst[(size_t)b * cap + i] >= ep_pair ? i : -1);
            int d = 0;
            longlong2 x = make_longlong2(0, 0);
            if (u >= 0) {
                const longlong2 r = A.root[u];
                x = meet(r, __ldcg(F + (dense ? u : slot_find(sh, false, u))));
                d = (x.x != r.x || x.y != r.y) ? 1 : 0;
            }
            sh.scan[tid] = d;
            __syncthreads();
            for (int o = 1; o < kPThreads; o <<= 1) {
                const int y = tid >= o ? sh.scan[tid - o] : 0;
                __syncthreads();
                sh.scan[tid] += y;
                __syncthreads();
            }
            if (d) {
                const long long pos = (long long)wbase + written + sh.scan[tid] - 1;
                if (pos < A.ecap) {
                    A.evar[pos] = u;
                    A.el[pos] = kdec(x.x);
                    A.eu[pos] = kdec(x.y);
                }
            }
            written += sh.scan[kPThreads - 1];
            __syncthreads();
        }
        }
        // reset the touched slots of the branch to neutral
        for (int i = tid; i < nt; i += kPThreads) {
            const int u = tl[i];
            Sb(b, 0)[u] = neutral_keys();
            Sb(b, 1)[u] = neutral_keys();
        }
        __syncthreads();
    }
    if (!dense) {
        // free the pair's slots (after both branches' outputs, which look variables up)
        for (int b = 0; b < 2; ++b)
            for (int i = tid; i < sh.ntouch[b]; i += kPThreads) sh.hkey[touched[(size_t)b * cap + i]] = 0;
        __syncthreads();
    }
}

// The pairs that the sparse pass left (their branches touched more variables than a table
// holds), with dense scratch `slot`: taken from the overflow list one at a time until it is
// empty.  The slot's epoch counter and the block's are combined by maximum, so the stamps in
// the slot's scratch and in the block's row state keep growing.
__device__ void dense_drain(ProbeShared& sh, const DevProblem& P, const ProbeArgs& A, int slot) {
    const int tid = threadIdx.x;
    const size_t n = (size_t)P.n;
    unsigned long long* rw = A.rw + (size_t)blockIdx.x * P.m;
    int* wl = A.wl + (size_t)blockIdx.x * 2 * P.m;
    const PairScratch ds{P.n, A.Sd + (size_t)slot * 4 * n, A.vstd + (size_t)slot * 2 * n, A.chgd + (size_t)slot * 4 * n,
                         A.touchedd + (size_t)slot * 2 * n};
    // nothing listed (the usual case): no epoch exchange
    if (tid == 0) sh.last = __ldcg(A.ovf_ctr) < __ldcg(A.novf);
    __syncthreads();
    const bool work = sh.last;
    __syncthreads();
    if (!work) return;
    if (tid == 0) {
        const unsigned long long e = __ldcg(A.epd + slot);
        if (e > sh.ep) sh.ep = e;
    }
    for (;;) {
        if (tid == 0) {
            int got = -1;
            for (;;) {
                const int c = __ldcg(A.ovf_ctr);
                if (c >= __ldcg(A.novf)) break;
                if (atomicCAS(A.ovf_ctr, c, c + 1) != c) continue;
                // the entry's writer took its index just before writing it
                const long long t0 = clock64();
                int v;
                while ((v = reinterpret_cast<volatile int*>(A.ovf)[c]) < 0) {
                    if (clock64() - t0 > kPSpinLimit) {
                        atomicExch(A.error, 2);
                        break;
                    }
                }
                A.ovf[c] = -1;
                got = v;
                break;
            }
            sh.pair = got;
            sh.ep_pair = ++sh.ep;
            sh.hfull = 0;
        }
        __syncthreads();
        const int pair = sh.pair;
        if (pair < 0) break;
        probe_pair(sh, P, A, ds, rw, wl, pair, true);
    }
    if (tid == 0) A.epd[slot] = sh.ep;
    __syncthreads();
}

// Exclusive prefix sums of the branches' entry counts into offsets[0..nb] and the total, by one
// block of kPThreads threads: 4 consecutive counts per thread per tile, shuffle scans within and
// across the warps.
__device__ void block_offsets(int nb, const long long* ecount, int64_t* offsets, unsigned long long* total) {
    __shared__ long long wsum[kPWarps];
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    long long carry = 0;
    for (int base = 0; base < nb; base += 4 * kPThreads) {
        const int i0 = base + 4 * t;
        long long v[4], own = 0;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            v[k] = i0 + k < nb ? __ldcg(ecount + i0 + k) : 0;
            own += v[k];
        }
        long long x = own;
        for (int o = 1; o < 32; o <<= 1) {
            const long long y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wsum[w] = x;
        __syncthreads();
        long long before = 0, all = 0;
        for (int q = 0; q < kPWarps; ++q) {
            if (q < w) before += wsum[q];
            all += wsum[q];
        }
        long long ex = carry + before + x - own;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (i0 + k < nb) offsets[i0 + k] = (int64_t)ex;
            ex += v[k];
        }
        carry += all;
        __syncthreads();
    }
    if (t == 0) {
        offsets[nb] = (int64_t)carry;
        *total = (unsigned long long)carry;
    }
}

// Sparse pass over every pair of the batch, then the dense pass over the pairs it left: blocks
// that own a dense scratch take those listed so far, and the last block to finish takes the rest
// and then writes every branch's entry offset.
__global__ void __launch_bounds__(kPThreads, kPBlocksPerSM) probe_kernel(DevProblem P, ProbeArgs A) {
    __shared__ ProbeShared sh;
    const int tid = threadIdx.x;
    const PairScratch hs{kHCap, A.S + (size_t)blockIdx.x * 4 * kHCap, A.vst + (size_t)blockIdx.x * 2 * kHCap,
                         A.chg + (size_t)blockIdx.x * 4 * kHCap, A.touched + (size_t)blockIdx.x * 2 * kHCap};
    for (int i = tid; i < kHCapMax; i += kPThreads) sh.hkey[i] = 0;
    // the block's epoch counter: in shared memory during the launch (thread 0 only), stored
    // back at the end so that the next launch continues from it
    if (tid == 0) sh.ep = A.ep[blockIdx.x];
    __syncthreads();
    for (;;) {
        if (tid == 0) {
            sh.pair = atomicAdd(A.pair_ctr, 1);
            sh.ep_pair = ++sh.ep;
            sh.hfull = 0;
        }
        __syncthreads();
        const int pair = sh.pair;
        if (pair >= A.npairs) break;
        probe_pair(sh, P, A, hs, A.rw + (size_t)blockIdx.x * P.m, A.wl + (size_t)blockIdx.x * 2 * P.m, pair, false);
    }
    if ((int)blockIdx.x < A.dense_blocks) dense_drain(sh, P, A, blockIdx.x);
    __syncthreads();
    if (tid == 0) sh.last = atom_add_acqrel_u32(reinterpret_cast<unsigned*>(A.done), 1u) == gridDim.x - 1;
    __syncthreads();
    const bool last = sh.last;
    __syncthreads();   // every thread has read the flag before the drain reuses it
    if (last) {
        dense_drain(sh, P, A, (int)blockIdx.x < A.dense_blocks ? blockIdx.x : 0);
        block_offsets(2 * A.npairs, A.ecount, A.offsets, A.ectr);
    }
    if (tid == 0) A.ep[blockIdx.x] = sh.ep;
}

__global__ void k_root_keys(int n, const double* lb, const double* ub, const unsigned char* is_int, longlong2* out) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
        out[v] = normalized_keys(lb[v], ub[v], is_int[v] != 0);
}

__global__ void k_fill_neutral(size_t count, longlong2* S) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x)
        S[i] = neutral_keys();
}

// offsets (exclusive scan of the entry counts) and the copy of every branch's entries to its
// place, in branch order; one block, the counts are few
// copy of every branch's entries to the cache, launched before the host knows the total: it
// does nothing when the total passes the cache's capacity (the call then reports BP_ERR_CAPACITY)
__global__ void k_probe_copy(int nb, const long long* ecount, const long long* estart, const int64_t* offsets,
                             const unsigned long long* total, long long cap,
                             const int* tv, const double* tl, const double* tu, int* ov, double* ol, double* ou) {
    if ((long long)*total > cap) return;
    const int lane = threadIdx.x & 31;
    for (int b = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; b < nb; b += (gridDim.x * blockDim.x) >> 5) {
        const long long c = ecount[b], s = estart[b], o = offsets[b];
        for (long long i = lane; i < c; i += 32) {
            ov[o + i] = tv[s + i];
            ol[o + i] = tl[s + i];
            ou[o + i] = tu[s + i];
        }
    }
}

// normalised keys of caller bounds (device arrays) into out
int root_keys(mip_problem* p, const double* lb, const double* ub, longlong2* out, cudaStream_t s) {
    if (p->n) {
        const int g = (p->n + 255) / 256 < 1216 ? (p->n + 255) / 256 : 1216;
        k_root_keys<<<g, 256, 0, s>>>(p->n, lb, ub, p->dp.is_int, out);
        BP_CUDA_TRY(cudaGetLastError());
    }
    return BP_OK;
}

struct ProbeWork {
    int blocks = 0;
    int glanes = 32;
    longlong2* S = nullptr;
    unsigned long long* vst = nullptr;
    unsigned long long* rw = nullptr;
    int* wl = nullptr;
    int* chg = nullptr;
    int* touched = nullptr;
    int dense_blocks = 0;        // blocks of the dense pass, with their own per-variable scratch
    longlong2* Sd = nullptr;
    unsigned long long* vstd = nullptr;
    int* chgd = nullptr;
    int* touchedd = nullptr;
    int* ovf = nullptr;          // pairs left to the dense pass (capacity cap_branches / 2)
    unsigned long long* ep = nullptr;
    int* ctr = nullptr;          // [0] next pair, [1] pairs left to the dense pass, [2] next of
                                 // those, [3] blocks done with the sparse pass
    unsigned long long* epd = nullptr;
    unsigned long long* ectr = nullptr;
    long long* ecount = nullptr;
    long long* estart = nullptr;
    int cap_branches = 0;
    int* tv = nullptr;
    double* tl = nullptr;
    double* tu = nullptr;
    long long tcap = 0;
    float* rowcap = nullptr;     // m
};

// Lanes per worklist row in the probe kernel: with kPLane nonzeros per lane, a group of G lanes
// covers 4 G nonzeros per segment; rows of a probe are few per round, so the narrowest group whose
// segment holds the average row (with room for its spread) keeps the most rows in flight.
static int probe_group_lanes(int m, long long nnz) {
    const double avg = m ? (double)nnz / m : 0.0;
    if (avg <= 0.5 * 8 * kPLane) return 8;
    if (avg <= 0.75 * 16 * kPLane) return 16;
    return 32;
}

static ProbeWork* probe_work(mip_problem* p) { return static_cast<ProbeWork*>(p->probe_work); }

static void probe_work_free(mip_problem* p) {
    delete probe_work(p);   // device buffers are in p->allocs
    p->probe_work = nullptr;
}

static int probe_prepare(mip_problem* p, int nbranches, long long cap, cudaStream_t s) {
    if (!p->probe_work) {
        ProbeWork* pw = new ProbeWork();
        p->probe_work = pw;
        p->free_hooks[0] = probe_work_free;
        int sms = 0;
        BP_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->device));
        // sparse pass: kPBlocksPerSM blocks per SM (fewer when their scratch, 104 kHCap + 16 m
        // bytes each, would pass the budget; at least one per SM), each with a table of kHCap
        // slots; dense pass: as many blocks as kPDenseBudget holds at 104 n bytes each (at least
        // one, at most the sparse pass's), sharing the row state of the sparse blocks
        const size_t per_block = 104 * (size_t)kHCap + 16 * (size_t)p->m + 64;
        size_t nb = (size_t)kPBlocksPerSM * sms;
        if (nb * per_block > kPScratchBudget) nb = kPScratchBudget / per_block;
        if (nb < (size_t)sms) nb = (size_t)sms;
        pw->blocks = (int)nb;
        size_t nd = kPDenseBudget / (104 * (size_t)p->n + 64);
        if (nd < 1) nd = 1;
        if (nd > nb) nd = nb;
        pw->dense_blocks = (int)nd;
        const size_t B = (size_t)pw->blocks, D = nd, H = (size_t)kHCap, n = (size_t)p->n, m = (size_t)p->m;
        BP_TRY(dalloc(p, &pw->S, B * 4 * H));
        BP_TRY(dalloc(p, &pw->vst, B * 2 * H));
        BP_TRY(dalloc(p, &pw->chg, B * 4 * H));
        BP_TRY(dalloc(p, &pw->touched, B * 2 * H));
        BP_TRY(dalloc(p, &pw->Sd, D * 4 * n));
        BP_TRY(dalloc(p, &pw->vstd, D * 2 * n));
        BP_TRY(dalloc(p, &pw->chgd, D * 4 * n));
        BP_TRY(dalloc(p, &pw->touchedd, D * 2 * n));
        BP_TRY(dalloc(p, &pw->rw, B * m));
        BP_TRY(dalloc(p, &pw->wl, B * 2 * m));
        BP_TRY(dalloc(p, &pw->ep, B));
        BP_TRY(dalloc(p, &pw->ctr, 4));
        BP_TRY(dalloc(p, &pw->epd, D));
        BP_CUDA_TRY(cudaMemsetAsync(pw->epd, 0, sizeof(unsigned long long) * D, s));
        BP_TRY(dalloc(p, &pw->ectr, 2));
        BP_TRY(dalloc(p, &pw->rowcap, m));
        k_fill_neutral<<<1024, 256, 0, s>>>(B * 4 * H, pw->S);
        if (D * 4 * n) k_fill_neutral<<<1024, 256, 0, s>>>(D * 4 * n, pw->Sd);
        BP_CUDA_TRY(cudaGetLastError());

        pw->glanes = GPUBP_PROBE_GLANES ? GPUBP_PROBE_GLANES : probe_group_lanes(p->m, p->nnz);
    }
    ProbeWork* pw = probe_work(p);
    if (nbranches > pw->cap_branches) {
        BP_TRY(dalloc(p, &pw->ecount, (size_t)nbranches));
        BP_TRY(dalloc(p, &pw->estart, (size_t)nbranches));
        BP_TRY(dalloc(p, &pw->ovf, (size_t)nbranches / 2 + 1));
        BP_CUDA_TRY(cudaMemsetAsync(pw->ovf, 0xff, sizeof(int) * ((size_t)nbranches / 2 + 1), s));
        pw->cap_branches = nbranches;
    }
    if (cap > pw->tcap) {
        BP_TRY(dalloc(p, &pw->tv, (size_t)cap));
        BP_TRY(dalloc(p, &pw->tl, (size_t)cap));
        BP_TRY(dalloc(p, &pw->tu, (size_t)cap));
        pw->tcap = cap;
    }
    return BP_OK;
}

// ------------------------------------------------------------------ cache application
// Global bounds from a probing cache (Section 2.2): each pair's two branch boxes cover the
// probed variable's integer domain, so every solution lies in a feasible branch's implied box
// (the root bounds where the branch lists nothing); the bounds are intersected, pair by pair,
// with the hull of the feasible branches' boxes.  Bounds are ordered keys, so every
// intersection is an atomicMax / atomicMin and the pairs apply in any order.
struct ApplyCtl {
    int first_pair, first_var, fixed_pairs, pad;
    unsigned long long tightened;
};

__global__ void k_apply_init(int n, const double* lb, const double* ub, const unsigned char* is_int, longlong2* K,
                             ApplyCtl* ctl) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x)
        K[j] = normalized_keys(lb[j], ub[j], is_int[j] != 0);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        ctl->first_pair = INT_MAX;
        ctl->first_var = INT_MAX;
        ctl->fixed_pairs = 0;
        ctl->tightened = 0;
    }
}

// One warp per pair.  Both branches feasible: each entry of branch 0 looks its variable up in
// branch 1's entries (both ascend by variable) and a variable listed by both gets the hull.
__global__ void k_apply_pairs(int npairs, const int32_t* status, const int64_t* off, const int32_t* ev,
                              const double* el, const double* eu, longlong2* K, ApplyCtl* ctl) {
    const int lane = threadIdx.x & 31;
    for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < npairs; i += (gridDim.x * blockDim.x) >> 5) {
        const bool f0 = status[2 * i] != BP_INFEASIBLE, f1 = status[2 * i + 1] != BP_INFEASIBLE;
        if (!f0 && !f1) {
            if (lane == 0) atomicMin(&ctl->first_pair, i);
            continue;
        }
        if (f0 != f1) {
            const int e = 2 * i + (f0 ? 0 : 1);
            if (lane == 0) atomicAdd(&ctl->fixed_pairs, 1);
            for (long long q = off[e] + lane; q < off[e + 1]; q += 32) {
                const int w = ev[q];
                atomicMax(&K[w].x, dkey(el[q]));
                atomicMin(&K[w].y, dkey(eu[q]));
            }
            continue;
        }
        const long long b0 = off[2 * i + 1], b1 = off[2 * i + 2];
        for (long long q = off[2 * i] + lane; q < b0; q += 32) {
            const int w = ev[q];
            long long lo = b0, hi = b1;   // first entry of branch 1 with variable >= w
            while (lo < hi) {
                const long long mid = (lo + hi) >> 1;
                if (ev[mid] < w) lo = mid + 1;
                else hi = mid;
            }
            if (lo < b1 && ev[lo] == w) {
                atomicMax(&K[w].x, dkey(fmin(el[q], el[lo])));
                atomicMin(&K[w].y, dkey(fmax(eu[q], eu[lo])));
            }
        }
    }
}

__global__ void k_apply_finish(int n, double* lb, double* ub, const unsigned char* is_int, const longlong2* K,
                               ApplyCtl* ctl) {
    const int lane = threadIdx.x & 31;
    for (int jb = blockIdx.x * blockDim.x; jb < n; jb += gridDim.x * blockDim.x) {
        const int j = jb + threadIdx.x;
        bool changed = false;
        if (j < n) {
            const bool ii = is_int[j] != 0;
            const longlong2 k = K[j];
            const longlong2 in = normalized_keys(lb[j], ub[j], ii);
            changed = k.x != in.x || k.y != in.y;
            lb[j] = kdec(k.x);
            ub[j] = kdec(k.y);
            if (crossed(ii, k.x, k.y)) atomicMin(&ctl->first_var, j);
        }
        const unsigned m = __ballot_sync(0xffffffffu, changed);
        if (lane == 0 && m) atomicAdd(&ctl->tightened, (unsigned long long)__popc(m));
    }
}

static bool probe_scratch_ready(const mip_problem* p, int nbranches, long long cap) {
    const ProbeWork* pw = static_cast<const ProbeWork*>(p->probe_work);
    return pw && nbranches <= pw->cap_branches && cap <= pw->tcap;
}

}  // namespace gpubp

using namespace gpubp;

extern "C" int probe_cache_apply(mip_problem* p, double* lb, double* ub, int32_t npairs, const probe_cache* cache,
                                 probe_apply_result* result, void* stream) {
    if (!p || !result || npairs < 0 || (p->n && (!lb || !ub)) ||
        (npairs && (!cache || !cache->status || !cache->offsets))) {
        set_error("probe_cache_apply: null or negative argument");
        return BP_ERR_INVALID;
    }
    cudaStream_t s = (cudaStream_t)stream;
    Work& w = p->w;
    if (!w.aux) BP_TRY(dalloc(p, &w.aux, 4));
    ApplyCtl* ctl = reinterpret_cast<ApplyCtl*>(w.aux);
    longlong2* K = w.bkey[1];
    const int n = p->n;
    const int gn = (n + 255) / 256 < 1216 ? ((n + 255) / 256 > 0 ? (n + 255) / 256 : 1) : 1216;
    k_apply_init<<<gn, 256, 0, s>>>(n, lb, ub, p->dp.is_int, K, ctl);
    BP_CUDA_TRY(cudaGetLastError());
    if (npairs) {
        const int gp = (npairs * 32 + 255) / 256 < 1216 ? (npairs * 32 + 255) / 256 : 1216;
        k_apply_pairs<<<gp, 256, 0, s>>>(npairs, cache->status, cache->offsets, cache->ent_var, cache->ent_l,
                                         cache->ent_u, K, ctl);
        BP_CUDA_TRY(cudaGetLastError());
    }
    k_apply_finish<<<gn, 256, 0, s>>>(n, lb, ub, p->dp.is_int, K, ctl);
    BP_CUDA_TRY(cudaGetLastError());
    ApplyCtl h;
    BP_CUDA_TRY(cudaMemcpyAsync(&h, ctl, sizeof(h), cudaMemcpyDeviceToHost, s));
    BP_CUDA_TRY(cudaStreamSynchronize(s));
    p->last_stream = s;
    result->first_infeasible_pair = h.first_pair == INT_MAX ? -1 : h.first_pair;
    result->first_infeasible_var = h.first_var == INT_MAX ? -1 : h.first_var;
    result->fixed_pairs = h.fixed_pairs;
    result->tightened = (int64_t)h.tightened;
    result->status = (h.first_pair != INT_MAX || h.first_var != INT_MAX) ? BP_INFEASIBLE : BP_FIXPOINT;
    return BP_OK;
}

extern "C" int bp_probe_batch_async(mip_problem* p, const double* root_lb, const double* root_ub, int32_t npairs,
                                    const int32_t* var, const double* boxes, const bp_params* params,
                                    probe_cache* cache, int64_t* status_dev, void* stream);

extern "C" int bp_probe_batch(mip_problem* p, const double* root_lb, const double* root_ub, int32_t npairs,
                              const int32_t* var, const double* boxes, const bp_params* params, probe_cache* cache,
                              void* stream) {
    if (!p || !cache) {
        set_error("bp_probe_batch: null argument");
        return BP_ERR_INVALID;
    }
    cudaStream_t s = (cudaStream_t)stream;
    Work& w = p->w;
    if (!w.aux) BP_TRY(dalloc(p, &w.aux, 4));
    int64_t* words_dev = reinterpret_cast<int64_t*>(w.aux) + 2;
    cache->needed = 0;
    BP_TRY(bp_probe_batch_async(p, root_lb, root_ub, npairs, var, boxes, params, cache, words_dev, stream));
    int64_t words[2] = {0, 0};   // entry total and the index check, read together
    BP_CUDA_TRY(cudaMemcpyAsync(words, words_dev, sizeof(words), cudaMemcpyDeviceToHost, s));
    BP_CUDA_TRY(cudaStreamSynchronize(s));
    if (words[1] == 2) {
        set_error("bp_probe_batch: a bounded device wait ran out");
        return BP_ERR_TIMEOUT;
    }
    if (words[1]) {
        set_error("bp_probe_batch: a variable index is outside [0, n)");
        return BP_ERR_INVALID;
    }
    cache->needed = words[0];
    if (words[0] > cache->cap) {
        set_error("probing cache needs %lld entries, capacity %lld", (long long)words[0], (long long)cache->cap);
        return BP_ERR_CAPACITY;
    }
    return BP_OK;
}

extern "C" int bp_probe_batch_async(mip_problem* p, const double* root_lb, const double* root_ub, int32_t npairs,
                                    const int32_t* var, const double* boxes, const bp_params* params,
                                    probe_cache* cache, int64_t* status_dev, void* stream) {
    if (!p || !cache || !status_dev || npairs < 0 || (npairs && (!var || !boxes)) ||
        (p->n && (!root_lb || !root_ub))) {
        set_error("bp_probe_batch: null or negative argument");
        return BP_ERR_INVALID;
    }
    if ((npairs && (!cache->status || !cache->rounds || !cache->nnz_updates || !cache->offsets)) || cache->cap < 0 ||
        (cache->cap > 0 && (!cache->ent_var || !cache->ent_l || !cache->ent_u))) {
        set_error("bp_probe_batch: cache arrays missing");
        return BP_ERR_INVALID;
    }
    bp_params prm;
    if (params) prm = *params;
    else bp_params_default(&prm);
    if (!(prm.theta >= 0.0) || prm.max_rounds < 0) {
        set_error("bp_probe_batch: invalid parameters");
        return BP_ERR_INVALID;
    }
    cudaStream_t s = (cudaStream_t)stream;
    if (npairs == 0) {
        BP_CUDA_TRY(cudaMemsetAsync(status_dev, 0, 2 * sizeof(int64_t), s));
        if (cache->offsets) BP_CUDA_TRY(cudaMemsetAsync(cache->offsets, 0, sizeof(int64_t), s));
        return BP_OK;
    }
    const long long cap = cache->cap > 0 ? cache->cap : 1;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    BP_CUDA_TRY(cudaStreamIsCapturing(s, &cs));
    if (cs != cudaStreamCaptureStatusNone && !probe_scratch_ready(p, 2 * npairs, cap)) {
        set_error("bp_probe_batch_async: the probing scratch for %d pairs and %lld cache entries is not allocated; "
                  "make one call of this size before capturing",
                  npairs, cap);
        return BP_ERR_INVALID;
    }
    BP_TRY(probe_prepare(p, 2 * npairs, cap, s));
    ProbeWork* pw = probe_work(p);
    longlong2* root = p->w.bkey[0];
    BP_TRY(root_keys(p, root_lb, root_ub, root, s));
    {
        const int rows_per_block = 8 * (32 / pw->glanes);
        const int g = p->m / rows_per_block + 1 < 1216 ? p->m / rows_per_block + 1 : 1216;
        k_probe_rowcap<<<g, 256, 0, s>>>(p->dp, root, pw->rowcap, pw->ctr, pw->ectr, pw->glanes);
        BP_CUDA_TRY(cudaGetLastError());
    }
    ProbeArgs a;
    a.root = root;
    a.rowcap = pw->rowcap;
    a.var = var;
    a.boxes = boxes;
    a.npairs = npairs;
    a.S = pw->S;
    a.vst = pw->vst;
    a.rw = pw->rw;
    a.wl = pw->wl;
    a.chg = pw->chg;
    a.touched = pw->touched;
    a.ep = pw->ep;
    a.pair_ctr = pw->ctr;
    a.ovf = pw->ovf;
    a.novf = pw->ctr + 1;
    a.ovf_ctr = pw->ctr + 2;
    a.done = pw->ctr + 3;
    a.dense_blocks = pw->dense_blocks;
    a.Sd = pw->Sd;
    a.vstd = pw->vstd;
    a.chgd = pw->chgd;
    a.touchedd = pw->touchedd;
    a.epd = pw->epd;
    a.glanes = pw->glanes;
    a.theta = prm.theta;
    a.max_rounds = prm.max_rounds;
    a.status = cache->status;
    a.rounds = cache->rounds;
    a.nnzu = cache->nnz_updates;
    a.ecount = pw->ecount;
    a.offsets = cache->offsets;
    a.estart = pw->estart;
    a.evar = pw->tv;
    a.el = pw->tl;
    a.eu = pw->tu;
    a.ectr = pw->ectr;
    a.ecap = pw->tcap;
    a.error = reinterpret_cast<int*>(pw->ectr + 1);
    probe_kernel<<<pw->blocks, kPThreads, 0, s>>>(p->dp, a);
    BP_CUDA_TRY(cudaGetLastError());
    const int nb = 2 * npairs;
    k_probe_copy<<<(nb * 32 + 255) / 256 < 1216 ? (nb * 32 + 255) / 256 : 1216, 256, 0, s>>>(
        nb, pw->ecount, pw->estart, cache->offsets, pw->ectr, cache->cap, pw->tv, pw->tl, pw->tu, cache->ent_var,
        cache->ent_l, cache->ent_u);
    BP_CUDA_TRY(cudaGetLastError());
    // the entry total and the index check go to the caller's device words: no synchronisation
    BP_CUDA_TRY(cudaMemcpyAsync(status_dev, pw->ectr, 2 * sizeof(int64_t), cudaMemcpyDeviceToDevice, s));
    p->last_stream = s;
    return BP_OK;
}
