// The local search's move scoring (Section 2.4, the paper's GPU Local-MIP): the mixed-tight-move
// core under a weighted violation F = sum_k w_k max(0, (A x)_k - g_k), and its objective moves
// (Local-MIP's lift and breakthrough moves under a weighted objective row).
//
// A candidate is, for a violated row and a variable in it, the value that alone satisfies the
// row (integers by the smallest integer step, clamped to the bounds), scored by the drop of F
// over the variable's column (rows ascending); the best (largest score; ties: smallest variable,
// smallest value, then a mixed tight move before a breakthrough move) moves when its score is
// positive, otherwise every violated row's weight grows by 1.
//
// local_search_mtm keeps every candidate's score in a slot per nonzero and, after a move,
// recomputes only the moved variable's distance-2 neighbourhood (the paper's neighbour lists,
// found on the fly), all of it after a weight bump; the iterations run in one persistent
// cooperative launch (k_ls_loop: selection, the move by block 0, the neighbourhood update,
// separated by grid barriers).
//
// local_search_objective recomputes every score each iteration (D = c x - c x* enters every
// score), five launches per iteration:
//   k_lso_lift        at a point with no violated row: the point is copied out when it becomes
//                     the incumbent, and a thread per variable with a cost forms its lift move
//                     (as far against the cost's sign as every row of its column allows);
//   k_lso_lift_apply  one block: records the incumbent (D restarts at 0) and applies the best
//                     lift move when its gain is positive, which ends the iteration;
//   k_ls_score        a warp per violated row, lanes over its nonzeros, each candidate scored by
//                     a walk of its column; a thread per costed variable adds the objective
//                     row's tight values (breakthrough) while that row is violated; every score
//                     adds the objective row's weighted drop; one best key per block;
//   k_ls_apply        one block: the best over the blocks (a total order, so the result does
//                     not depend on the reduction's order); the move and its column's activity
//                     updates, or the weights are to grow (w0 when no row is violated);
//   k_ls_bump         every violated row's weight grows by 1.
// Everything stays on the device (no host read per iteration).  The activities start from a
// thread-per-row sum in row order and are updated in the order of the moves as compensated
// (Kahan) sums, one compensation term per row, summed afresh every recompute_period iterations
// (Local-MIP's numerics), so the search is bit-for-bit that of a sequential implementation with
// the same operation order.
#include <climits>
#include <cstdlib>
#include <cmath>

#include "bp_host.h"

namespace gpubp {

constexpr int kLsThreads = 256;
constexpr int kLsLongRow = 256;   // longer rows are scanned by the whole grid, not one thread or warp
constexpr int kLsRedBlocks = 304;

struct LsKey {
    double score;
    double t;
    int j;
    int kind;   // 0: a mixed tight move, 1: a breakthrough move (the objective row's tight move)
};

__device__ __forceinline__ LsKey ls_none() { return LsKey{-INFINITY, INFINITY, INT_MAX, 2}; }

// a before b: larger score; ties: smaller variable, smaller value, then the smaller kind
__device__ __forceinline__ bool ls_before(const LsKey& a, const LsKey& b) {
    if (a.score != b.score) return a.score > b.score;
    if (a.j != b.j) return a.j < b.j;
    if (a.t != b.t) return a.t < b.t;
    return a.kind < b.kind;
}

__device__ __forceinline__ LsKey ls_shfl(const LsKey& k, int lane) {
    LsKey o;
    o.score = __shfl_sync(0xffffffffu, k.score, lane);
    o.t = __shfl_sync(0xffffffffu, k.t, lane);
    o.j = __shfl_sync(0xffffffffu, k.j, lane);
    o.kind = __shfl_sync(0xffffffffu, k.kind, lane);
    return o;
}

struct LsCtl {
    int nviol;        // violated rows seen by this iteration's scoring pass
    int bump;         // the weights grow in this iteration
    int moves, bumps;
    int moved_j;      // the variable this iteration moved, -1 if none
    unsigned bar_count;   // arrivals at the persistent search's grid barriers
    int error;            // a barrier wait gave up
    int nbr_count;        // rows of the moved variable's column
    int nbr_total;        // their entries, in one flat sequence
    // objective moves
    int nv;           // violated rows of the current point (kept through every move)
    int has_best;     // an incumbent exists
    int done;         // a lift move ended this iteration
    int lifts, breakthroughs, improvements;
    int cost_any, cost_frac;   // some cost is nonzero / some nonzero cost is not integral on an integer
    double D;         // c x - c x* since the incumbent was recorded
    double w0;        // the objective row's weight
    double delta;     // the objective row's step
};

// L = A x in row order; with nv, the violated rows are counted too
__global__ void k_ls_activities(DevProblem P, const double* __restrict__ x, double* __restrict__ L, int* nv) {
    int cnt = 0;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < P.m; k += gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int q = P.row_ptr[k]; q < P.row_ptr[k + 1]; ++q) s = __dadd_rn(s, __dmul_rn(P.val[q], x[P.col[q]]));
        L[k] = s;
        const double g = P.grow[k].x;
        if (isfinite(g) && __dsub_rn(s, g) > 0.0) ++cnt;
    }
    if (nv) {
        cnt = __reduce_add_sync(0xffffffffu, cnt);
        if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(nv, cnt);
    }
}

// ceil(e / c) for e > 0, c > 0, corrected to the exact quotient's ceiling for integers
__device__ __forceinline__ double ls_ceil_div(double e, double c) {
    double d = ceil(__ddiv_rn(e, c));
    if (e == floor(e) && c == floor(c)) {
        for (int it = 0; it < 4 && d > 1.0 && __dmul_rn(d - 1.0, c) >= e; ++it) d -= 1.0;
        for (int it = 0; it < 4 && __dmul_rn(d, c) < e; ++it) d += 1.0;
    }
    return d;
}

// floor(e / c) for e >= 0, c > 0, corrected to the exact quotient's floor for integers
__device__ __forceinline__ double ls_floor_div(double e, double c) {
    double d = floor(__ddiv_rn(e, c));
    if (e == floor(e) && c == floor(c)) {
        for (int it = 0; it < 4 && __dmul_rn(d + 1.0, c) <= e; ++it) d += 1.0;
        for (int it = 0; it < 4 && d > 0.0 && __dmul_rn(d, c) > e; ++it) d -= 1.0;
    }
    return d;
}

// the value that alone removes violation v > 0 of a row with coefficient a on x_j
__device__ __forceinline__ double ls_tight(double xj, double a, double v, bool integer) {
    if (integer) {
        const double d = ls_ceil_div(v, fabs(a));
        return a > 0.0 ? __dsub_rn(xj, d) : __dadd_rn(xj, d);
    }
    return __dsub_rn(xj, __ddiv_rn(v, a));
}

// loads of the data that moves during a search (activities, weights, points, cached slots):
// through L2 (CG) inside the persistent search, where other blocks wrote it since the last
// barrier; plain loads between launches
template <bool CG, typename Tp>
__device__ __forceinline__ Tp ls_ld(const Tp* p) {
    if constexpr (CG) return __ldcg(p);
    else return *p;
}

// the drop of the weighted row violation if x_j alone moves by dx: the column's rows in order,
// the loads of four entries issued together
template <bool CG = false>
__device__ __forceinline__ double ls_column_score(const DevProblem& P, const double* __restrict__ w,
                                                  const double* __restrict__ L, int j, double dx) {
    double s = 0.0;
    const int cb = P.col_ptr[j], ce = P.col_ptr[j + 1];
    for (int c0 = cb; c0 < ce; c0 += 4) {
        int rr[4];
        double gg[4], ll[4], ww[4], aa[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) rr[i] = c0 + i < ce ? P.row_idx[c0 + i] : -1;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int r = rr[i] >= 0 ? rr[i] : 0;
            gg[i] = P.grow[r].x;
            ll[i] = ls_ld<CG>(L + r);
            ww[i] = ls_ld<CG>(w + r);
            aa[i] = c0 + i < ce ? P.col_val[c0 + i] : 0.0;
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            if (rr[i] < 0 || !isfinite(gg[i])) continue;
            const double o = __dsub_rn(ll[i], gg[i]);
            const double nw = __dsub_rn(__dadd_rn(ll[i], __dmul_rn(aa[i], dx)), gg[i]);
            const double ov = o > 0.0 ? o : 0.0, nv = nw > 0.0 ? nw : 0.0;
            s = __dadd_rn(s, __dmul_rn(ww[i], __dsub_rn(ov, nv)));
        }
    }
    return s;
}

// the objective row's weighted drop: w0 (max(0, D + delta) - max(0, (D + c_j dx) + delta))
__device__ __forceinline__ double ls_objective_term(double D, double delta, double w0, double cj, double dx) {
    const double o = __dadd_rn(D, delta);
    const double nw = __dadd_rn(__dadd_rn(D, __dmul_rn(cj, dx)), delta);
    const double ov = o > 0.0 ? o : 0.0, nv = nw > 0.0 ? nw : 0.0;
    return __dmul_rn(w0, __dsub_rn(ov, nv));
}

template <bool OBJ>
__global__ void __launch_bounds__(kLsThreads) k_ls_score(DevProblem P, const double* __restrict__ lb,
                                                         const double* __restrict__ ub, const double* __restrict__ x,
                                                         const double* __restrict__ w, const double* __restrict__ L,
                                                         LsKey* __restrict__ part, LsCtl* ctl,
                                                         const double* __restrict__ cost) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    bool with_obj = false;
    double D = 0.0, delta = 0.0, w0 = 0.0;
    if constexpr (OBJ) {
        if (ctl->done) return;   // a lift move ended this iteration
        with_obj = ctl->has_best != 0;
        D = ctl->D;
        delta = ctl->delta;
        w0 = ctl->w0;
    }
    LsKey best = ls_none();
    int nviol = 0;
    for (int k = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; k < P.m; k += (gridDim.x * blockDim.x) >> 5) {
        const double g = P.grow[k].x;
        if (!isfinite(g)) continue;
        const double v = __dsub_rn(L[k], g);
        if (!(v > 0.0)) continue;
        ++nviol;
        for (int q = P.row_ptr[k] + lane; q < P.row_ptr[k + 1]; q += 32) {
            const int j = P.col[q];
            const double a = P.val[q], xj = x[j];
            double t = ls_tight(xj, a, v, P.is_int[j] != 0);
            t = t < lb[j] ? lb[j] : t;   // max(t, l), then min(., u)
            t = t > ub[j] ? ub[j] : t;
            if (t == xj) continue;
            const double dx = __dsub_rn(t, xj);
            double s = ls_column_score(P, w, L, j, dx);
            if (OBJ && with_obj) s = __dadd_rn(s, ls_objective_term(D, delta, w0, cost[j], dx));
            const LsKey key{s, t, j, 0};
            if (ls_before(key, best)) best = key;
        }
    }
    if constexpr (OBJ) {
        // breakthrough moves: the objective row's tight values while it is violated
        const double v0 = __dadd_rn(D, delta);
        if (with_obj && v0 > 0.0) {
            for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < P.n; j += gridDim.x * blockDim.x) {
                const double cj = cost[j];
                if (cj == 0.0) continue;
                const double xj = x[j];
                double t = ls_tight(xj, cj, v0, P.is_int[j] != 0);
                t = t < lb[j] ? lb[j] : t;
                t = t > ub[j] ? ub[j] : t;
                if (t == xj) continue;
                const double dx = __dsub_rn(t, xj);
                const double s = __dadd_rn(ls_column_score(P, w, L, j, dx), ls_objective_term(D, delta, w0, cj, dx));
                const LsKey key{s, t, j, 1};
                if (ls_before(key, best)) best = key;
            }
        }
    }
    // warp, then block reduction of the keys; violated rows counted once per warp
    for (int o = 16; o > 0; o >>= 1) {
        const LsKey other = ls_shfl(best, lane ^ o);
        if (ls_before(other, best)) best = other;
    }
    __shared__ LsKey wk[kLsThreads / 32];
    __shared__ int wn[kLsThreads / 32];
    if (lane == 0) {
        wk[wid] = best;
        wn[wid] = nviol;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        LsKey b = wk[0];
        int nv = wn[0];
        for (int i = 1; i < kLsThreads / 32; ++i) {
            if (ls_before(wk[i], b)) b = wk[i];
            nv += wn[i];
        }
        part[blockIdx.x] = b;
        if (nv) atomicAdd(&ctl->nviol, nv);
    }
}

// one block moves x_j to t: the activities of its column, then x_j (and, with the objective
// moves, D and the count of violated rows)
// the activity update of a move: L_r += a dx as a compensated (Kahan) sum with the row's
// compensation term C_r
template <bool OBJ, bool CG = false, int NT = kLsThreads>
__device__ void ls_move(const DevProblem& P, double* __restrict__ x, double* __restrict__ L, double* __restrict__ C,
                        int j, double t, LsCtl* ctl, const double* __restrict__ cost) {
    __shared__ int sdv[NT / 32];
    const double dx = __dsub_rn(t, ls_ld<CG>(x + j));
    int dv = 0;
    for (int c = P.col_ptr[j] + threadIdx.x; c < P.col_ptr[j + 1]; c += NT) {
        const int r = P.row_idx[c];
        const double old = ls_ld<CG>(L + r);
        const double y = __dsub_rn(__dmul_rn(P.col_val[c], dx), ls_ld<CG>(C + r));
        const double nw = __dadd_rn(old, y);
        C[r] = __dsub_rn(__dsub_rn(nw, old), y);
        L[r] = nw;
        if constexpr (OBJ) {
            const double g = P.grow[r].x;
            if (isfinite(g)) dv += (__dsub_rn(nw, g) > 0.0 ? 1 : 0) - (__dsub_rn(old, g) > 0.0 ? 1 : 0);
        }
    }
    if constexpr (OBJ) {
        dv = __reduce_add_sync(0xffffffffu, dv);
        if ((threadIdx.x & 31) == 0) sdv[threadIdx.x >> 5] = dv;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if constexpr (OBJ) {
            int tot = 0;
            for (int i = 0; i < NT / 32; ++i) tot += sdv[i];
            ctl->nv += tot;
            ctl->D = __dadd_rn(ctl->D, __dmul_rn(cost[j], dx));
        }
        x[j] = t;
        ctl->moves += 1;
    }
}

// the best of the per-block keys, in every thread
__device__ LsKey ls_block_best(const LsKey* __restrict__ part, int nparts) {
    __shared__ LsKey sk[kLsThreads];
    LsKey b = ls_none();
    for (int i = threadIdx.x; i < nparts; i += kLsThreads)
        if (ls_before(part[i], b)) b = part[i];
    sk[threadIdx.x] = b;
    __syncthreads();
    for (int o = kLsThreads / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o && ls_before(sk[threadIdx.x + o], sk[threadIdx.x])) sk[threadIdx.x] = sk[threadIdx.x + o];
        __syncthreads();
    }
    const LsKey best = sk[0];
    __syncthreads();
    return best;
}

template <bool OBJ>
__global__ void __launch_bounds__(kLsThreads) k_ls_apply(DevProblem P, double* __restrict__ x, double* __restrict__ L,
                                                         double* __restrict__ C, const LsKey* __restrict__ part,
                                                         int nparts, LsCtl* ctl, const double* __restrict__ cost) {
    if constexpr (OBJ) {
        if (ctl->done) {   // a lift move ended this iteration
            __syncthreads();
            if (threadIdx.x == 0) {
                ctl->done = 0;
                ctl->bump = 0;
                ctl->nviol = 0;
            }
            return;
        }
    }
    const LsKey best = ls_block_best(part, nparts);
    const int nviol = OBJ ? ctl->nv : ctl->nviol;
    __syncthreads();
    if (best.j != INT_MAX && best.score > 0.0) {
        ls_move<OBJ>(P, x, L, C, best.j, best.t, ctl, cost);
        if (threadIdx.x == 0) {
            ctl->bump = 0;
            ctl->moved_j = best.j;
            if (OBJ) ctl->breakthroughs += best.kind;
        }
    } else if (threadIdx.x == 0) {
        ctl->moved_j = -1;
        ctl->bump = nviol > 0 ? 1 : 0;
        if (nviol > 0) {
            ctl->bumps += 1;
        } else if (OBJ && ctl->has_best) {   // no violated row: the objective row's weight grows
            ctl->w0 = __dadd_rn(ctl->w0, 1.0);
            ctl->bumps += 1;
        }
    }
    if (threadIdx.x == 0) ctl->nviol = 0;
}

// the lift moves at a point with no violated row; the point is copied to x_best first when it
// becomes the incumbent (the first such point, or D < 0)
__global__ void __launch_bounds__(kLsThreads) k_lso_lift(DevProblem P, const double* __restrict__ lb,
                                                         const double* __restrict__ ub, const double* __restrict__ x,
                                                         const double* __restrict__ L, const double* __restrict__ cost,
                                                         double* __restrict__ x_best, LsKey* __restrict__ part,
                                                         const LsCtl* ctl) {
    if (ctl->nv != 0) return;
    const bool rec = !ctl->has_best || ctl->D < 0.0;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    LsKey best = ls_none();
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < P.n; j += gridDim.x * blockDim.x) {
        const double xj = x[j];
        if (rec) x_best[j] = xj;
        const double cj = cost[j];
        if (cj == 0.0) continue;
        const bool up = cj < 0.0;   // the direction sigma = -sign(c_j)
        const bool integer = P.is_int[j] != 0;
        double step = INFINITY;
        for (int c = P.col_ptr[j]; c < P.col_ptr[j + 1]; ++c) {
            const double a = P.col_val[c];
            if (up ? !(a > 0.0) : !(a < 0.0)) continue;
            const int r = P.row_idx[c];
            const double g = P.grow[r].x;
            if (!isfinite(g)) continue;
            const double slack = __dsub_rn(g, L[r]);
            const double sr = integer ? ls_floor_div(slack, fabs(a)) : __ddiv_rn(slack, fabs(a));
            step = sr < step ? sr : step;
        }
        double t;
        if (isinf(step)) {
            t = up ? ub[j] : lb[j];
        } else {
            t = up ? __dadd_rn(xj, step) : __dsub_rn(xj, step);
            t = t < lb[j] ? lb[j] : t;
            t = t > ub[j] ? ub[j] : t;
        }
        if (!isfinite(t) || t == xj) continue;
        const double gain = -__dmul_rn(cj, __dsub_rn(t, xj));
        const LsKey key{gain, t, j, 0};
        if (ls_before(key, best)) best = key;
    }
    for (int o = 16; o > 0; o >>= 1) {
        const LsKey other = ls_shfl(best, lane ^ o);
        if (ls_before(other, best)) best = other;
    }
    __shared__ LsKey wk[kLsThreads / 32];
    if (lane == 0) wk[wid] = best;
    __syncthreads();
    if (threadIdx.x == 0) {
        LsKey b = wk[0];
        for (int i = 1; i < kLsThreads / 32; ++i)
            if (ls_before(wk[i], b)) b = wk[i];
        part[blockIdx.x] = b;
    }
}

// records the incumbent, then applies the best lift move when its gain is positive
__global__ void __launch_bounds__(kLsThreads) k_lso_lift_apply(DevProblem P, double* __restrict__ x,
                                                               double* __restrict__ L, double* __restrict__ C,
                                                               const LsKey* __restrict__ part, int nparts, LsCtl* ctl,
                                                               const double* __restrict__ cost) {
    const int nv = ctl->nv;
    const bool rec = nv == 0 && (!ctl->has_best || ctl->D < 0.0);
    __syncthreads();
    if (threadIdx.x == 0) {
        ctl->done = 0;
        if (rec) {
            ctl->has_best = 1;
            ctl->D = 0.0;
            ctl->improvements += 1;
        }
    }
    if (nv != 0) return;
    const LsKey best = ls_block_best(part, nparts);
    if (best.j != INT_MAX && best.score > 0.0) {
        ls_move<true>(P, x, L, C, best.j, best.t, ctl, cost);
        if (threadIdx.x == 0) {
            ctl->lifts += 1;
            ctl->done = 1;
        }
    }
}

// the objective row's step: 1 when every nonzero cost sits on an integer variable and is
// integral, else 1e-4
__global__ void k_lso_cost_flags(DevProblem P, const double* __restrict__ cost, LsCtl* ctl) {
    int any = 0, frac = 0;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < P.n; j += gridDim.x * blockDim.x) {
        const double cj = cost[j];
        if (cj == 0.0) continue;
        any = 1;
        if (!P.is_int[j] || cj != floor(cj)) frac = 1;
    }
    any = __reduce_or_sync(0xffffffffu, any);
    frac = __reduce_or_sync(0xffffffffu, frac);
    if ((threadIdx.x & 31) == 0) {
        if (any) atomicOr(&ctl->cost_any, 1);
        if (frac) atomicOr(&ctl->cost_frac, 1);
    }
}

__global__ void k_lso_init(LsCtl* ctl, double w0) {
    ctl->delta = ctl->cost_any && !ctl->cost_frac ? 1.0 : 1e-4;
    ctl->w0 = w0;
    ctl->D = 0.0;
}

// ---- the score cache of the mixed-tight-move search (distance-2 neighbourhood updates) ----
//
// The candidate of violated row k on the variable of its nonzero q is kept in slot q: its value
// T[q] and score S[q] (-inf: no candidate).  A slot depends on row k's activity, on x_j and on
// the activities and weights of the rows of column j.  A move of x_j* changes x_j* and the
// activities of the rows of column j* only, so the slots that change are those (k, j) with j
// in a row of column j* (the distance-2 neighbourhood of j*): the persistent search recomputes
// exactly those, with the same function, so every score equals a full recomputation bit for
// bit.  A weight bump changes every slot: all are recomputed.

// CSC entry -> CSR position: each nonzero finds its row in its column's ascending row list
__global__ void k_ls_perm(DevProblem P, int* __restrict__ perm) {
    const int lane = threadIdx.x & 31;
    for (int k = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; k < P.m; k += (gridDim.x * blockDim.x) >> 5) {
        for (int q = P.row_ptr[k] + lane; q < P.row_ptr[k + 1]; q += 32) {
            const int j = P.col[q];
            int lo = P.col_ptr[j], hi = P.col_ptr[j + 1] - 1;
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (P.row_idx[mid] < k) lo = mid + 1;
                else hi = mid;
            }
            perm[lo] = q;
        }
    }
}

// the slot of row k (violation v > 0) on variable j with coefficient a
template <bool CG = false>
__device__ __forceinline__ void ls_slot(const DevProblem& P, const double* __restrict__ lb,
                                        const double* __restrict__ ub, const double* __restrict__ x,
                                        const double* __restrict__ w, const double* __restrict__ L, int j, double a,
                                        double v, double* __restrict__ T, double* __restrict__ S, int q) {
    const double xj = ls_ld<CG>(x + j);
    double t = ls_tight(xj, a, v, P.is_int[j] != 0);
    t = t < lb[j] ? lb[j] : t;
    t = t > ub[j] ? ub[j] : t;
    if (t == xj) {
        S[q] = -INFINITY;
        return;
    }
    S[q] = ls_column_score<CG>(P, w, L, j, __dsub_rn(t, xj));
    T[q] = t;
}

// the rows longer than kLsLongRow (their order does not matter: every reduction over them is
// under a total order)
__global__ void k_ls_long_rows(DevProblem P, int* __restrict__ list, int* __restrict__ count) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < P.m; k += gridDim.x * blockDim.x)
        if (P.row_ptr[k + 1] - P.row_ptr[k] > kLsLongRow) list[atomicAdd(count, 1)] = k;
}

// every slot of every violated row (at the start; after a weight bump the persistent search
// does the same): a warp per row, and the long rows' slots over the whole grid
__global__ void __launch_bounds__(kLsThreads) k_ls_full(DevProblem P, const double* __restrict__ lb,
                                                        const double* __restrict__ ub, const double* __restrict__ x,
                                                        const double* __restrict__ w, const double* __restrict__ L,
                                                        double* __restrict__ T, double* __restrict__ S,
                                                        const int* __restrict__ long_list,
                                                        const int* __restrict__ long_count) {
    const int lane = threadIdx.x & 31;
    for (int k = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; k < P.m; k += (gridDim.x * blockDim.x) >> 5) {
        const double g = P.grow[k].x;
        if (!isfinite(g)) continue;
        const double v = __dsub_rn(L[k], g);
        if (!(v > 0.0)) continue;
        const int qb = P.row_ptr[k], qe = P.row_ptr[k + 1];
        if (qe - qb > kLsLongRow) continue;
        for (int q = qb + lane; q < qe; q += 32) ls_slot(P, lb, ub, x, w, L, P.col[q], P.val[q], v, T, S, q);
    }
    const int nl = *long_count;
    for (int i = 0; i < nl; ++i) {
        const int k = long_list[i];
        const double g = P.grow[k].x;
        if (!isfinite(g)) continue;
        const double v = __dsub_rn(L[k], g);
        if (!(v > 0.0)) continue;
        for (int q = P.row_ptr[k] + blockIdx.x * blockDim.x + threadIdx.x; q < P.row_ptr[k + 1];
             q += gridDim.x * blockDim.x)
            ls_slot(P, lb, ub, x, w, L, P.col[q], P.val[q], v, T, S, q);
    }
}

// ---- the whole mixed-tight-move search in one persistent cooperative launch ----
//
// One block per SM: the three grid barriers of an iteration cost less with fewer arrivals on
// their counter (knapsack/cover, 1M nonzeros, 256-thread blocks: 0.049 ms per iteration with
// 152 blocks, 0.053 with 304, 0.088 with every resident block; 0.062 as five launches per
// iteration; 1,024-thread blocks: 0.089).
// Per iteration: selection over the cached slots (a thread per row, so a warp checks 32 rows
// at once and each violated row's slots are read by its own thread), a grid barrier, the move
// or the bump decision by block 0, a grid barrier, then the neighbourhood update: the entries
// of the rows of column j*, taken as one flat sequence, spread over the grid's warps (a dense
// row spreads over the whole grid, short rows run side by side), each warp's lanes over the
// variable's column (a slot reached through several rows is written with the same value); or,
// after a bump, the weights, a barrier and the full recomputation; a grid barrier.  Every load
// of moving data goes through L2.

constexpr long long kLsSpinLimit = 4000000000LL;   // clock64 cycles (about 2 s) per barrier wait

// every block arrives once on a count that only grows; the wait is a bounded spin of acquire
// loads (a timeout sets the error word, and every block leaves the search at its next check)
__device__ __forceinline__ bool ls_grid_sync(LsCtl* ctl, unsigned& bar_k) {
    __syncthreads();
    if (threadIdx.x == 0) {
        atom_add_acqrel_u32(&ctl->bar_count, 1u);
        const unsigned target = gridDim.x * (bar_k + 1u);
        const long long t0 = clock64();
        while (ld_acquire_u32(&ctl->bar_count) < target) {
            if (clock64() - t0 > kLsSpinLimit) {
                atomicExch(&ctl->error, 1);
                break;
            }
        }
    }
    bar_k += 1u;
    __syncthreads();
    return __ldcg(&ctl->error) == 0;
}

// every slot of every violated row, inside the persistent search: a warp per row, the long
// rows' slots over the whole grid
__device__ void ls_all_slots(const DevProblem& P, const double* __restrict__ lb, const double* __restrict__ ub,
                             const double* __restrict__ x, const double* __restrict__ w,
                             const double* __restrict__ L, double* __restrict__ T, double* __restrict__ S,
                             const int* __restrict__ long_list, int nlong, int gw, int nw, int lane, int tid,
                             int nthr) {
    for (int k = gw; k < P.m; k += nw) {
        const double g = P.grow[k].x;
        if (!isfinite(g)) continue;
        const double v = __dsub_rn(L[k], g);
        if (!(v > 0.0)) continue;
        const int qb = P.row_ptr[k], qe = P.row_ptr[k + 1];
        if (qe - qb > kLsLongRow) continue;
        for (int q = qb + lane; q < qe; q += 32) ls_slot<false>(P, lb, ub, x, w, L, P.col[q], P.val[q], v, T, S, q);
    }
    for (int i = 0; i < nlong; ++i) {
        const int k = long_list[i];
        const double g = P.grow[k].x;
        if (!isfinite(g)) continue;
        const double v = __dsub_rn(L[k], g);
        if (!(v > 0.0)) continue;
        for (int q = P.row_ptr[k] + tid; q < P.row_ptr[k + 1]; q += nthr)
            ls_slot<false>(P, lb, ub, x, w, L, P.col[q], P.val[q], v, T, S, q);
    }
}

constexpr int kLsLoopThreads = 256;
constexpr int kLsNbrStaged = 1024;   // rows of the moved column staged in shared memory

__global__ void __launch_bounds__(kLsLoopThreads) k_ls_loop(DevProblem P, const double* __restrict__ lb,
                                                        const double* __restrict__ ub, double* __restrict__ x,
                                                        double* __restrict__ w, double* __restrict__ L,
                                                        double* __restrict__ T, double* __restrict__ S,
                                                        const int* __restrict__ perm, LsKey* __restrict__ part,
                                                        int* __restrict__ nbr_row, int* __restrict__ nbr_start,
                                                        const int* __restrict__ long_list,
                                                        const int* __restrict__ long_count, double* __restrict__ C,
                                                        LsCtl* ctl, int it0, int iterations, int recompute_period,
                                                        int skip_block) {
    __shared__ int s_row[kLsNbrStaged], s_start[kLsNbrStaged];
    __shared__ int s_wsum[kLsLoopThreads / 32];
    __shared__ int s_carry;
    __shared__ LsKey wk[kLsLoopThreads / 32];
    __shared__ int wn[kLsLoopThreads / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int tid = blockIdx.x * blockDim.x + threadIdx.x, nthr = gridDim.x * blockDim.x;
    const int gw = tid >> 5, nw = nthr >> 5;
    const int nlong = *long_count;
    unsigned bar_k = 0;
    for (int it = 0; it < iterations; ++it) {
        if (skip_block == (int)blockIdx.x) {
            // test-only failure: this block stops arriving at the grid barriers, so the others'
            // bounded waits run out and the call reports BP_ERR_TIMEOUT
            return;
        }
        if (recompute_period > 0 && it0 + it > 0 && (it0 + it) % recompute_period == 0) {
            // the activities summed afresh in row order, the compensation cleared, then every
            // violated row's slots
            for (int k = tid; k < P.m; k += nthr) {
                double sum = 0.0;
                for (int q = P.row_ptr[k]; q < P.row_ptr[k + 1]; ++q)
                    sum = __dadd_rn(sum, __dmul_rn(P.val[q], x[P.col[q]]));
                L[k] = sum;
                C[k] = 0.0;
            }
            if (!ls_grid_sync(ctl, bar_k)) return;
            ls_all_slots(P, lb, ub, x, w, L, T, S, long_list, nlong, gw, nw, lane, tid, nthr);
            if (!ls_grid_sync(ctl, bar_k)) return;
        }
        // selection: the best cached key of the violated rows
        LsKey best = ls_none();
        int nviol = 0;
        for (int k = tid; k < P.m; k += nthr) {
            const double g = P.grow[k].x;
            if (!isfinite(g) || !(__dsub_rn(L[k], g) > 0.0)) continue;
            ++nviol;
            const int qb = P.row_ptr[k], qe = P.row_ptr[k + 1];
            if (qe - qb > kLsLongRow) continue;   // scanned below by the whole grid
            for (int q0 = qb; q0 < qe; q0 += 4) {
                double sc[4], tt[4];
                int jj[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int q = q0 + i < qe ? q0 + i : q0;
                    sc[i] = S[q];
                    tt[i] = T[q];
                    jj[i] = P.col[q];
                }
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    if (q0 + i >= qe || sc[i] == -INFINITY) continue;
                    const LsKey key{sc[i], tt[i], jj[i], 0};
                    if (ls_before(key, best)) best = key;
                }
            }
        }
        for (int i = 0; i < nlong; ++i) {
            const int k = long_list[i];
            const double g = P.grow[k].x;
            if (!isfinite(g) || !(__dsub_rn(L[k], g) > 0.0)) continue;
            for (int q = P.row_ptr[k] + tid; q < P.row_ptr[k + 1]; q += nthr) {
                const double sc = S[q];
                if (sc == -INFINITY) continue;
                const LsKey key{sc, T[q], P.col[q], 0};
                if (ls_before(key, best)) best = key;
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const LsKey other = ls_shfl(best, lane ^ o);
            if (ls_before(other, best)) best = other;
        }
        nviol = __reduce_add_sync(0xffffffffu, nviol);
        if (lane == 0) {
            wk[wid] = best;
            wn[wid] = nviol;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            LsKey b = wk[0];
            int nv = wn[0];
            for (int i = 1; i < kLsLoopThreads / 32; ++i) {
                if (ls_before(wk[i], b)) b = wk[i];
                nv += wn[i];
            }
            part[blockIdx.x] = b;
            if (nv) atomicAdd(&ctl->nviol, nv);
        }
        if (!ls_grid_sync(ctl, bar_k)) return;
        // block 0: the best over the blocks; the move, or the bump decision
        if (blockIdx.x == 0) {
            __shared__ LsKey sk[kLsLoopThreads];
            LsKey b = ls_none();
            for (int i = threadIdx.x; i < (int)gridDim.x; i += kLsLoopThreads) {
                const LsKey pk{__ldcg(&part[i].score), __ldcg(&part[i].t), __ldcg(&part[i].j), 0};
                if (ls_before(pk, b)) b = pk;
            }
            sk[threadIdx.x] = b;
            __syncthreads();
            for (int o = kLsLoopThreads / 2; o > 0; o >>= 1) {
                if (threadIdx.x < o && ls_before(sk[threadIdx.x + o], sk[threadIdx.x]))
                    sk[threadIdx.x] = sk[threadIdx.x + o];
                __syncthreads();
            }
            const LsKey bb = sk[0];
            const int nv = __ldcg(&ctl->nviol);
            __syncthreads();
            if (bb.j != INT_MAX && bb.score > 0.0) {
                ls_move<false, false, kLsLoopThreads>(P, x, L, C, bb.j, bb.t, ctl, nullptr);
                // the rows of column j* and the starts of their entries in one flat sequence
                // (a block-wide exclusive scan of the row lengths)
                const int cb = P.col_ptr[bb.j], cn = P.col_ptr[bb.j + 1] - cb;
                if (threadIdx.x == 0) s_carry = 0;
                __syncthreads();
                for (int base = 0; base < cn; base += kLsLoopThreads) {
                    const int i = base + threadIdx.x;
                    int r = 0, len = 0;
                    if (i < cn) {
                        r = P.row_idx[cb + i];
                        len = P.row_ptr[r + 1] - P.row_ptr[r];
                    }
                    int v = len;
                    for (int o = 1; o < 32; o <<= 1) {
                        const int u = __shfl_up_sync(0xffffffffu, v, o);
                        if (lane >= o) v += u;
                    }
                    if (lane == 31) s_wsum[wid] = v;
                    __syncthreads();
                    if (wid == 0) {
                        int ws = lane < kLsLoopThreads / 32 ? s_wsum[lane] : 0;
                        for (int o = 1; o < 32; o <<= 1) {
                            const int u = __shfl_up_sync(0xffffffffu, ws, o);
                            if (lane >= o) ws += u;
                        }
                        if (lane < kLsLoopThreads / 32) s_wsum[lane] = ws;
                    }
                    __syncthreads();
                    if (i < cn) {
                        nbr_row[i] = r;
                        nbr_start[i] = s_carry + (wid ? s_wsum[wid - 1] : 0) + v - len;
                    }
                    __syncthreads();
                    if (threadIdx.x == 0) s_carry += s_wsum[kLsLoopThreads / 32 - 1];
                    __syncthreads();
                }
                if (threadIdx.x == 0) {
                    ctl->bump = 0;
                    ctl->moved_j = bb.j;
                    ctl->nbr_count = cn;
                    ctl->nbr_total = s_carry;
                }
            } else if (threadIdx.x == 0) {
                ctl->moved_j = -1;
                ctl->bump = nv > 0 ? 1 : 0;
                if (nv > 0) ctl->bumps += 1;
            }
            if (threadIdx.x == 0) ctl->nviol = 0;
        }
        if (!ls_grid_sync(ctl, bar_k)) return;
        const int bump = __ldcg(&ctl->bump), js = __ldcg(&ctl->moved_j);
        if (bump) {
            for (int k = tid; k < P.m; k += nthr) {
                const double g = P.grow[k].x;
                if (isfinite(g) && __dsub_rn(L[k], g) > 0.0) w[k] = __dadd_rn(w[k], 1.0);
            }
            if (!ls_grid_sync(ctl, bar_k)) return;
            ls_all_slots(P, lb, ub, x, w, L, T, S, long_list, nlong, gw, nw, lane, tid, nthr);
        } else if (js >= 0) {
            const int cn = __ldcg(&ctl->nbr_count), E = __ldcg(&ctl->nbr_total);
            const bool staged = cn <= kLsNbrStaged;
            if (staged)
                for (int i = threadIdx.x; i < cn; i += kLsLoopThreads) {
                    s_row[i] = __ldcg(nbr_row + i);
                    s_start[i] = __ldcg(nbr_start + i);
                }
            __syncthreads();
            // flat entry f -> its row (the last with start <= f; empty rows are passed over)
            // and the variable there
            auto entry_var = [&](int f) -> int {
                int lo = 0, hi = cn - 1;
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    const int st = staged ? s_start[mid] : __ldcg(nbr_start + mid);
                    if (st <= f) lo = mid;
                    else hi = mid - 1;
                }
                const int r = staged ? s_row[lo] : __ldcg(nbr_row + lo);
                const int st = staged ? s_start[lo] : __ldcg(nbr_start + lo);
                return P.col[P.row_ptr[r] + (f - st)];
            };
            if (E <= 8 * nw) {
                // a warp per entry, its lanes over the variable's column
                for (int f = gw; f < E; f += nw) {
                    const int j = entry_var(f);
                    for (int c = P.col_ptr[j] + lane; c < P.col_ptr[j + 1]; c += 32) {
                        const int k = P.row_idx[c];
                        const double g = P.grow[k].x;
                        if (!isfinite(g)) continue;
                        const double v = __dsub_rn(L[k], g);
                        if (!(v > 0.0)) continue;
                        ls_slot<false>(P, lb, ub, x, w, L, j, P.col_val[c], v, T, S, perm[c]);
                    }
                }
            } else {
                // many entries (a dense row in the column): a thread per entry, its column in turn
                for (int f = tid; f < E; f += nthr) {
                    const int j = entry_var(f);
                    for (int c = P.col_ptr[j]; c < P.col_ptr[j + 1]; ++c) {
                        const int k = P.row_idx[c];
                        const double g = P.grow[k].x;
                        if (!isfinite(g)) continue;
                        const double v = __dsub_rn(L[k], g);
                        if (!(v > 0.0)) continue;
                        ls_slot<false>(P, lb, ub, x, w, L, j, P.col_val[c], v, T, S, perm[c]);
                    }
                }
            }
        }
        if (!ls_grid_sync(ctl, bar_k)) return;
    }
}

__global__ void k_ls_bump(DevProblem P, const double* __restrict__ L, double* __restrict__ w, const LsCtl* ctl) {
    if (!ctl->bump) return;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < P.m; k += gridDim.x * blockDim.x) {
        const double g = P.grow[k].x;
        if (isfinite(g) && __dsub_rn(L[k], g) > 0.0) w[k] = __dadd_rn(w[k], 1.0);
    }
}

// [0] violated rows, [1] sum of w_k v_k, [2] c^T x: block partial sums (fixed tree), then one
// block over the partials in block order
__global__ void __launch_bounds__(kLsThreads) k_ls_summary(DevProblem P, const double* c, const double* x,
                                                           const double* w, const double* L, double* part) {
    __shared__ double sh[3][kLsThreads];
    double v0 = 0.0, v1 = 0.0, v2 = 0.0;
    const int tid = blockIdx.x * blockDim.x + threadIdx.x, stride = gridDim.x * blockDim.x;
    for (int k = tid; k < P.m; k += stride) {
        const double g = P.grow[k].x;
        if (!isfinite(g)) continue;
        const double v = __dsub_rn(L[k], g);
        if (v > 0.0) {
            v0 += 1.0;
            v1 = __dadd_rn(v1, __dmul_rn(w[k], v));
        }
    }
    for (int j = tid; j < P.n; j += stride) v2 = __dadd_rn(v2, __dmul_rn(c[j], x[j]));
    sh[0][threadIdx.x] = v0;
    sh[1][threadIdx.x] = v1;
    sh[2][threadIdx.x] = v2;
    __syncthreads();
    for (int o = kLsThreads / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o)
            for (int i = 0; i < 3; ++i) sh[i][threadIdx.x] = __dadd_rn(sh[i][threadIdx.x], sh[i][threadIdx.x + o]);
        __syncthreads();
    }
    if (threadIdx.x < 3) part[3 * blockIdx.x + threadIdx.x] = sh[threadIdx.x][0];
}

__global__ void k_ls_summary_finish(const double* part, int nblocks, double* out) {
    if (threadIdx.x >= 3) return;
    double s = 0.0;
    for (int b = 0; b < nblocks; ++b) s = __dadd_rn(s, part[3 * b + threadIdx.x]);
    out[threadIdx.x] = s;
}

}  // namespace gpubp

using namespace gpubp;

namespace gpubp {

struct LsOut {
    double summary[6];   // violated rows, sum w_k v_k, c x; then the same for x_best
    LsCtl ctl;
};

// the search on the stream: `iterations` iterations from (x, w), the objective moves when OBJ
template <bool OBJ>
static int ls_run(mip_problem* p, const double* lb, const double* ub, double* x, double* w, double* x_best,
                  int iterations, int recompute_period, double w0, LsOut* out, cudaStream_t s) {
    void *pL = nullptr, *pC = nullptr, *pPart = nullptr, *pCtl = nullptr, *pSum = nullptr, *pOut = nullptr;
    void *pS = nullptr, *pT = nullptr, *pPerm = nullptr, *pNbr = nullptr, *pLong = nullptr;
    // the scoring passes on every resident block (their per-block bests are reduced by
    // k_ls_apply): k_ls_score with the objective moves, else the cache's first full pass
    static int occ_score[2] = {-1, -1}, occ_lift = -1;
    if (occ_score[OBJ] < 0) {
        cudaError_t oe = OBJ ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_score[OBJ], k_ls_score<OBJ>,
                                                                             kLsThreads, 0)
                             : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_score[OBJ], k_ls_full, kLsThreads, 0);
        if (oe != cudaSuccess) return fail_cuda(oe, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
    }

    if (OBJ && occ_lift < 0) {
        cudaError_t oe = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_lift, k_lso_lift, kLsThreads, 0);
        if (oe != cudaSuccess) return fail_cuda(oe, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
    }
    const int grid_score = p->sms * (occ_score[OBJ] > 0 ? occ_score[OBJ] : 1);
    const int grid_lift = p->sms * (occ_lift > 0 ? occ_lift : 1);
    const int grid_select = p->sms;   // the persistent search: one block per SM
    int nparts = grid_score > grid_lift ? grid_score : grid_lift;
    nparts = nparts > grid_select ? nparts : grid_select;
    auto release = [&]() {
        for (void* q : {pL, pC, pPart, pCtl, pSum, pOut, pS, pT, pPerm, pNbr, pLong})
            if (q) cudaFreeAsync(q, s);
    };
    cudaError_t e = cudaSuccess;
    const size_t nz = (size_t)(p->nnz ? p->nnz : 1);
    if (!OBJ && ((e = cudaMallocAsync(&pS, sizeof(double) * nz, s)) != cudaSuccess ||
                 (e = cudaMallocAsync(&pT, sizeof(double) * nz, s)) != cudaSuccess ||
                 (e = cudaMallocAsync(&pPerm, sizeof(int) * nz, s)) != cudaSuccess ||
                 (e = cudaMallocAsync(&pNbr, sizeof(int) * 2 * (size_t)(p->m + 1), s)) != cudaSuccess ||
                 (e = cudaMallocAsync(&pLong, sizeof(int) * (size_t)(p->m + 1), s)) != cudaSuccess)) {
        release();
        return fail_cuda(e, "cudaMallocAsync");
    }
    double* S = static_cast<double*>(pS);
    double* T = static_cast<double*>(pT);
    int* perm = static_cast<int*>(pPerm);
    int* nbr_row = static_cast<int*>(pNbr);
    int* nbr_start = nbr_row + (p->m + 1);
    int* long_count = static_cast<int*>(pLong);   // then the list of long rows
    int* long_list = long_count + 1;
    if ((e = cudaMallocAsync(&pL, sizeof(double) * (size_t)(p->m ? p->m : 1), s)) != cudaSuccess ||
        (e = cudaMallocAsync(&pC, sizeof(double) * (size_t)(p->m ? p->m : 1), s)) != cudaSuccess ||
        (e = cudaMallocAsync(&pPart, sizeof(LsKey) * (size_t)nparts, s)) != cudaSuccess ||
        (e = cudaMallocAsync(&pCtl, sizeof(LsCtl), s)) != cudaSuccess ||
        (e = cudaMallocAsync(&pSum, sizeof(double) * 3 * kLsRedBlocks, s)) != cudaSuccess ||
        (e = cudaMallocAsync(&pOut, sizeof(double) * 6, s)) != cudaSuccess) {
        release();
        return fail_cuda(e, "cudaMallocAsync");
    }
    double* L = static_cast<double*>(pL);
    double* C = static_cast<double*>(pC);   // the activities' compensation terms
    LsKey* part = static_cast<LsKey*>(pPart);
    LsCtl* ctl = static_cast<LsCtl*>(pCtl);
    double* sum = static_cast<double*>(pSum);
    double* dout = static_cast<double*>(pOut);
    const double* cost = p->obj;
    const int grid_rows = p->sms * 8;
    if ((e = cudaMemsetAsync(ctl, 0, sizeof(LsCtl), s)) != cudaSuccess ||
        (p->m && (e = cudaMemsetAsync(C, 0, sizeof(double) * (size_t)p->m, s)) != cudaSuccess)) {
        release();
        return fail_cuda(e, "cudaMemsetAsync");
    }
    k_ls_activities<<<grid_rows, kLsThreads, 0, s>>>(p->dp, x, L, OBJ ? &ctl->nv : nullptr);
    if (OBJ) {
        k_lso_cost_flags<<<grid_rows, kLsThreads, 0, s>>>(p->dp, cost, ctl);
        k_lso_init<<<1, 1, 0, s>>>(ctl, w0);
    }
    if (!OBJ && iterations > 0) {
        k_ls_perm<<<grid_rows, kLsThreads, 0, s>>>(p->dp, perm);
        if ((e = cudaMemsetAsync(long_count, 0, sizeof(int), s)) != cudaSuccess) {
            release();
            return fail_cuda(e, "cudaMemsetAsync");
        }
        k_ls_long_rows<<<grid_rows, kLsThreads, 0, s>>>(p->dp, long_list, long_count);
        k_ls_full<<<grid_score, kLsThreads, 0, s>>>(p->dp, lb, ub, x, w, L, T, S, long_list, long_count);
    }
    for (int it = 0; OBJ && it < iterations; ++it) {
        if (recompute_period > 0 && it > 0 && it % recompute_period == 0) {
            // the activities summed afresh in row order (violated rows counted again), the
            // compensation cleared
            if ((e = cudaMemsetAsync(&ctl->nv, 0, sizeof(int), s)) != cudaSuccess ||
                (e = cudaMemsetAsync(C, 0, sizeof(double) * (size_t)p->m, s)) != cudaSuccess) {
                release();
                return fail_cuda(e, "cudaMemsetAsync");
            }
            k_ls_activities<<<grid_rows, kLsThreads, 0, s>>>(p->dp, x, L, &ctl->nv);
        }
        k_lso_lift<<<grid_lift, kLsThreads, 0, s>>>(p->dp, lb, ub, x, L, cost, x_best, part, ctl);
        k_lso_lift_apply<<<1, kLsThreads, 0, s>>>(p->dp, x, L, C, part, grid_lift, ctl, cost);
        k_ls_score<OBJ><<<grid_score, kLsThreads, 0, s>>>(p->dp, lb, ub, x, w, L, part, ctl, cost);
        k_ls_apply<OBJ><<<1, kLsThreads, 0, s>>>(p->dp, x, L, C, part, grid_score, ctl, cost);
        k_ls_bump<<<grid_rows, kLsThreads, 0, s>>>(p->dp, L, w, ctl);
    }
    if (!OBJ && iterations > 0) {
        // launches of at most 2^16 iterations: at most four barriers per iteration keep the
        // arrival count (reset between launches) far from 32-bit wrap-around
        DevProblem dp = p->dp;
        // test-only failure injection: GPUBP_TEST_SKIP_BLOCK=b makes block b leave the search
        // without arriving at the grid barriers (the failure-detection tests; never set otherwise)
        const char* skip_env = getenv("GPUBP_TEST_SKIP_BLOCK");
        int skip = (skip_env && *skip_env) ? atoi(skip_env) : -1;
        for (int done = 0; done < iterations;) {
            int its = iterations - done < 65536 ? iterations - done : 65536;
            int it0 = done, rp = recompute_period;
            void* args[] = {&dp,        (void*)&lb,  (void*)&ub, &x,   &w,   &L,   &T,   &S,  &perm, &part,
                            &nbr_row,   &nbr_start,  &long_list, &long_count, &C, &ctl, &it0, &its, &rp, &skip};
            if ((done > 0 && (e = cudaMemsetAsync(&ctl->bar_count, 0, sizeof(unsigned), s)) != cudaSuccess) ||
                (e = cudaLaunchCooperativeKernel((const void*)k_ls_loop, dim3(grid_select), dim3(kLsLoopThreads), args, 0,
                                                 s)) != cudaSuccess) {
                release();
                return fail_cuda(e, "local search cooperative launch");
            }
            done += its;
        }
    }
    k_ls_summary<<<kLsRedBlocks, kLsThreads, 0, s>>>(p->dp, cost, x, w, L, sum);
    k_ls_summary_finish<<<1, 32, 0, s>>>(sum, kLsRedBlocks, dout);
    if (OBJ) {   // c x_best (the other two sums are not used)
        k_ls_summary<<<kLsRedBlocks, kLsThreads, 0, s>>>(p->dp, cost, x_best, w, L, sum);
        k_ls_summary_finish<<<1, 32, 0, s>>>(sum, kLsRedBlocks, dout + 3);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) {
        release();
        return fail_cuda(e, "local search launch");
    }
    e = cudaMemcpyAsync(out->summary, dout, sizeof(out->summary), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&out->ctl, ctl, sizeof(LsCtl), cudaMemcpyDeviceToHost, s);
    release();
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail_cuda(e, "local search results");
    p->last_stream = s;
    if (out->ctl.error) {
        set_error("local search: a grid barrier wait gave up");
        return BP_ERR_TIMEOUT;
    }
    return BP_OK;
}

}  // namespace gpubp

extern "C" int local_search_mtm(mip_problem* p, const double* lb, const double* ub, double* x, double* w,
                                const ls_params* params, ls_result* result, void* stream) {
    if (!p || !params || !result || (p->n && (!lb || !ub || !x)) || (p->m && !w)) {
        set_error("local_search_mtm: null argument");
        return BP_ERR_INVALID;
    }
    if (params->iterations < 0 || params->recompute_period < 0) {
        set_error("local_search_mtm: negative iteration count or recompute period");
        return BP_ERR_INVALID;
    }
    memset(result, 0, sizeof(*result));
    LsOut out;
    const int rc = ls_run<false>(p, lb, ub, x, w, nullptr, params->iterations, params->recompute_period, 0.0, &out,
                                 (cudaStream_t)stream);
    if (rc != BP_OK) return rc;
    result->iterations = params->iterations;
    result->moves = out.ctl.moves;
    result->bumps = out.ctl.bumps;
    result->violated = (int32_t)out.summary[0];
    result->weighted_violation = out.summary[1];
    result->objective = out.summary[2];
    return BP_OK;
}

extern "C" int local_search_objective(mip_problem* p, const double* lb, const double* ub, double* x, double* w,
                                      double* x_best, const ls_obj_params* params, ls_obj_result* result,
                                      void* stream) {
    if (!p || !params || !result || (p->n && (!lb || !ub || !x || !x_best)) || (p->m && !w)) {
        set_error("local_search_objective: null argument");
        return BP_ERR_INVALID;
    }
    if (params->iterations < 0 || params->recompute_period < 0 || !(params->obj_weight >= 0.0) ||
        !std::isfinite(params->obj_weight)) {
        set_error("local_search_objective: negative iteration count or invalid objective weight");
        return BP_ERR_INVALID;
    }
    memset(result, 0, sizeof(*result));
    LsOut out;
    const int rc =
        ls_run<true>(p, lb, ub, x, w, x_best, params->iterations, params->recompute_period, params->obj_weight, &out,
                     (cudaStream_t)stream);
    if (rc != BP_OK) return rc;
    result->iterations = params->iterations;
    result->moves = out.ctl.moves;
    result->bumps = out.ctl.bumps;
    result->violated = (int32_t)out.summary[0];
    result->weighted_violation = out.summary[1];
    result->objective = out.summary[2];
    result->lifts = out.ctl.lifts;
    result->breakthroughs = out.ctl.breakthroughs;
    result->improvements = out.ctl.improvements;
    result->found = out.ctl.has_best;
    result->best_objective = out.ctl.has_best ? out.summary[5] : INFINITY;
    result->obj_weight = out.ctl.w0;
    result->delta = out.ctl.delta;
    return BP_OK;
}
