// Bulk fix-and-propagate rounding (Section 2.3, Algorithm 1): fix_and_propagate.
//
// The loop itself is sequential (every bulk depends on the previous result), so the host
// drives the bulks and reads a few words per bulk for its control decisions; every step on the
// data runs in kernels: the list of unfixed variables, the implied-slack sums, the selection of
// the bulk (the first entries of the stable implied-slack order, selected, not sorted in full),
// the counter-based draws, the probing-cache conflict filter, the start boxes of the two
// candidate vectors, their propagations (the persistent engine, round 0 = rows of the variables
// the vector changes) and the final rounding.  The retry of a failed bulk one variable at a
// time runs on the device as a whole (without a probing cache): one persistent launch keeps
// the bounds as ordered keys and copies back only the variables each propagation changed.
//
// Random draws: splitmix64 (Steele, Lea, Flood, OOPSLA 2014) chained over (seed, bulk,
// variable, draw); the 53 high bits give a uniform double in [0, 1).
#include <climits>
#include <cmath>
#include <type_traits>
#include <vector>

#include "bp_host.h"
#include "fp_draw.cuh"

namespace gpubp {

// radix key of a double, ascending (descending when desc)
__device__ __forceinline__ unsigned long long fp_sort_key(double d, bool desc) {
    unsigned long long b = (unsigned long long)__double_as_longlong(d == 0.0 ? 0.0 : d);
    b = (b >> 63) ? ~b : (b | 0x8000000000000000ull);
    return desc ? ~b : b;
}

__global__ void k_intvars_flag(int n, const unsigned char* is_int, int* flag) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) flag[j] = is_int[j] ? 1 : 0;
}

__global__ void k_compact_idx(int n, const int* flag, const int* pos, int* out) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x)
        if (flag[j]) out[pos[j]] = j;
}

// initial order keys: pass 0 fractionality (ascending), pass 1 score (descending), pass 2 class
__global__ void k_initial_keys(int nint, const int* vars, const double* x, const double* l, const double* u,
                               const double* score, int which, unsigned long long* keys) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nint; i += gridDim.x * blockDim.x) {
        const int j = vars[i];
        if (which == 0) {
            const double xh = clampd(x[j], l[j], u[j]);
            const double f = __dsub_rn(xh, floor(xh));
            const double g = __dsub_rn(1.0, f);
            keys[i] = fp_sort_key(f < g ? f : g, false);
        } else if (which == 1) {
            keys[i] = fp_sort_key(score[j], true);
        } else {
            const double w = __dsub_rn(u[j], l[j]);
            keys[i] = w <= 1.0 ? 0ull : (w == 2.0 ? 1ull : 2ull);
        }
    }
}

__global__ void k_unset_flag(int nint, const int* order, const double* l, const double* u, int* flag) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nint; i += gridDim.x * blockDim.x) {
        const int j = order[i];
        flag[i] = l[j] < u[j] ? 1 : 0;
    }
}

__global__ void k_compact_list(int nint, const int* order, const int* flag, const int* pos, int* out) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nint; i += gridDim.x * blockDim.x)
        if (flag[i]) out[pos[i]] = order[i];
}

// row minimal activities (finite part, count of infinite terms) under bounds (l, u)
__global__ void k_row_act(DevProblem P, const double* l, const double* u, double* minfin, int* ninf) {
    const int lane = threadIdx.x & 31;
    for (int k = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; k < P.m; k += (gridDim.x * blockDim.x) >> 5) {
        double s = 0.0;
        int c = 0;
        for (int q = P.row_ptr[k] + lane; q < P.row_ptr[k + 1]; q += 32) {
            const double a = P.val[q];
            const double b = a > 0 ? l[P.col[q]] : u[P.col[q]];
            if (isinf(b)) ++c;
            else s = fma(a, b, s);
        }
        for (int o = 16; o > 0; o >>= 1) {
            s = __dadd_rn(s, __shfl_xor_sync(0xffffffffu, s, o));
            c += __shfl_xor_sync(0xffffffffu, c, o);
        }
        if (lane == 0) {
            minfin[k] = s;
            ninf[k] = c;
        }
    }
}

// implied slack S_i = sum over the variable's rows (ascending, as the transpose stores them)
// with a finite minimal activity of (a / max(g - L_min, tol))^2; keys descending
__global__ void k_implied_slack(DevProblem P, int cnt, const int* vars, const double* minfin, const int* ninf,
                                unsigned long long* keys) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += gridDim.x * blockDim.x) {
        const int j = vars[i];
        double S = 0.0;
        for (int s = P.col_ptr[j]; s < P.col_ptr[j + 1]; ++s) {
            const int k = P.row_idx[s];
            const double g = P.grow[k].x;
            if (isinf(g) || ninf[k]) continue;
            double slack = __dsub_rn(g, minfin[k]);
            if (slack < kTol) slack = kTol;
            const double sv = __ddiv_rn(P.col_val[s], slack);
            S = __dadd_rn(S, __dmul_rn(sv, sv));
        }
        keys[i] = fp_sort_key(S, true);
    }
}

__global__ void k_draws(int bsize, const int* bulk, const double* x, const double* l, const double* u,
                        unsigned long long seed, unsigned long long bulk_index, int single, const double* up_prob,
                        double* v0, double* v1) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < bsize; i += gridDim.x * blockDim.x) {
        const int j = bulk[i];
        const double xh = clampd(x[j], l[j], u[j]);
        const double a = clampd(draw_value(xh, seed, bulk_index, j, 0, up_prob), l[j], u[j]);
        double b;
        if (single) {
            const double fl = floor(xh);
            b = clampd(a == fl ? __dadd_rn(fl, 1.0) : fl, l[j], u[j]);
        } else {
            b = clampd(draw_value(xh, seed, bulk_index, j, 1, up_prob), l[j], u[j]);
        }
        v0[i] = a;
        v1[i] = b;
    }
}

__global__ void k_apply_plain(int bsize, const int* bulk, const double* v, double* cl, double* cu, int* kept) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < bsize; i += gridDim.x * blockDim.x) {
        const int j = bulk[i];
        cl[j] = v[i];
        cu[j] = v[i];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) *kept = bsize;
}

__device__ __forceinline__ bool var_crossed(bool is_i, double l, double u) {
    return is_i ? l > u : l > __dadd_rn(u, kTol);
}

// probing-cache conflict filter and warm start: one warp, the bulk in order; a fixing is kept
// if its value lies in the current box and its branch (when cached) is feasible and agrees
// with every bound implied so far; then the branch's implied bounds tighten the box
__global__ void k_apply_cache(int bsize, const int* bulk, const double* v, double* cl, double* cu,
                              const unsigned char* is_int, const int* pair_of, fp_cache c, int* kept) {
    const int lane = threadIdx.x;
    int nk = 0;
    for (int i = 0; i < bsize; ++i) {
        const int j = bulk[i];
        const double val = v[i];
        __syncwarp();
        if (!(val >= cl[j] && val <= cu[j])) continue;
        const int pi = pair_of[j];
        long long e = -1;
        if (pi >= 0) {
            for (int b = 0; b < 2; ++b) {
                const double lo = c.boxes[4 * pi + 2 * b], hi = c.boxes[4 * pi + 2 * b + 1];
                if (val >= lo && val <= hi) {
                    e = 2ll * pi + b;
                    break;
                }
            }
        }
        bool ok = true;
        if (e >= 0) {
            if (c.status[e] == BP_INFEASIBLE) ok = false;
            bool bad = false;
            if (ok) {
                for (long long q = c.offsets[e] + lane; q < c.offsets[e + 1]; q += 32) {
                    const int w = c.ent_var[q];
                    const double lo = c.ent_l[q] > cl[w] ? c.ent_l[q] : cl[w];
                    const double hi = c.ent_u[q] < cu[w] ? c.ent_u[q] : cu[w];
                    if (w == j ? !(val >= lo && val <= hi) : var_crossed(is_int[w] != 0, lo, hi)) bad = true;
                }
            }
            if (__any_sync(0xffffffffu, bad)) ok = false;
        }
        if (!ok) continue;
        ++nk;
        __syncwarp();
        if (lane == 0) {
            cl[j] = val;
            cu[j] = val;
        }
        __syncwarp();
        if (e >= 0) {
            for (long long q = c.offsets[e] + lane; q < c.offsets[e + 1]; q += 32) {
                const int w = c.ent_var[q];
                if (w == j) continue;
                if (c.ent_l[q] > cl[w]) cl[w] = c.ent_l[q];
                if (c.ent_u[q] < cu[w]) cu[w] = c.ent_u[q];
            }
        }
    }
    if (lane == 0) *kept = nk;
}

// variables whose start box differs from the current bounds (round 0 of the propagation),
// appended as off + j (the candidate's copy in the instance pair)
__global__ void k_diff(int n, const double* cl, const double* cu, const double* l, const double* u, int off,
                       int* list, int* count) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x)
        if (cl[j] != l[j] || cu[j] != u[j]) list[atomicAdd(count, 1)] = off + j;
}

// The two copies of a problem, block-diagonal: rows k and m + k, variables j and n + j.
__global__ void k_twin_arrays(DevProblem P, const double* lb, const double* ub, int64_t* rp, int* col, double* val,
                              double* g, double* l2, double* u2, unsigned char* is_int) {
    const long long m = P.m, n = P.n, nnz = P.nnz;
    const long long top = 2 * nnz > 2 * m + 1 ? (2 * nnz > 2 * n ? 2 * nnz : 2 * n) : (2 * m + 1 > 2 * n ? 2 * m + 1 : 2 * n);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < top; i += (long long)gridDim.x * blockDim.x) {
        if (i <= 2 * m) rp[i] = i < m ? P.row_ptr[i] : P.row_ptr[i - m] + nnz;
        if (i < 2 * m) g[i] = P.grow[i < m ? i : i - m].x;
        if (i < 2 * nnz) {
            const long long q = i < nnz ? i : i - nnz;
            col[i] = P.col[q] + (i < nnz ? 0 : (int)n);
            val[i] = P.val[q];
        }
        if (i < 2 * n) {
            const long long j = i < n ? i : i - n;
            l2[i] = lb[j];
            u2[i] = ub[j];
            is_int[i] = P.is_int[j];
        }
    }
}

static void twin_free(mip_problem* p) {
    if (p->twin) mip_free(p->twin);
    p->twin = nullptr;
}

// The instance pair on which both candidate vectors of a bulk propagate in one launch (built
// on first use, kept with the handle): the bulk's two propagations then share the launch, its
// grid barriers and its rounds, and each copy's status, rounds and nonzeros stay its own.
static int twin_problem(mip_problem* p, cudaStream_t s, mip_problem** out) {
    if (!p->twin) {
        if ((long long)p->nnz >= (1ll << 30) || p->m >= (1 << 30) || p->n >= (1 << 30)) {
            set_error("fix_and_propagate: the candidate pair holds two copies of the problem, so m, n and "
                      "nnz must each be below 2^30 (nnz = %lld)", (long long)p->nnz);
            return BP_ERR_CAPACITY;
        }
        const size_t m = (size_t)p->m, n = (size_t)p->n, nnz = (size_t)p->nnz;
        void* buf[7] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
        const size_t bytes[7] = {8 * (2 * m + 1), 4 * 2 * nnz + 4, 8 * 2 * nnz + 8, 8 * 2 * m + 8, 8 * 2 * n + 8,
                                 8 * 2 * n + 8, 2 * n + 1};
        int rc = BP_OK;
        for (int i = 0; i < 7 && rc == BP_OK; ++i)
            if (cudaMalloc(&buf[i], bytes[i]) != cudaSuccess) {
                set_error("fix_and_propagate: allocation of the instance pair failed");
                rc = BP_ERR_OOM;
            }
        mip_problem* t = nullptr;
        if (rc == BP_OK) {
            const long long top = 2 * (long long)(nnz > m + 1 ? (nnz > n ? nnz : n) : (m + 1 > n ? m + 1 : n));
            const int grid = (int)((top + 255) / 256 < 1216 ? (top + 255) / 256 : 1216);
            k_twin_arrays<<<grid > 0 ? grid : 1, 256, 0, s>>>(p->dp, p->def_lb, p->def_ub, (int64_t*)buf[0], (int*)buf[1],
                                                            (double*)buf[2], (double*)buf[3], (double*)buf[4],
                                                            (double*)buf[5], (unsigned char*)buf[6]);
            if (cudaGetLastError() != cudaSuccess) {
                set_error("fix_and_propagate: instance pair kernel failed to launch");
                rc = BP_ERR_CUDA;
            }
        }
        if (rc == BP_OK)
            rc = mip_load_csr(2 * p->m, 2 * p->n, (int64_t*)buf[0], (int*)buf[1], (double*)buf[2], (double*)buf[3],
                              (double*)buf[4], (double*)buf[5], (uint8_t*)buf[6], nullptr, BP_MEM_DEVICE, s, &t);
        cudaStreamSynchronize(s);
        for (void* b : buf)
            if (b) cudaFree(b);
        if (rc != BP_OK) return rc;
        const int32_t ro[3] = {0, p->m, 2 * p->m}, co[3] = {0, p->n, 2 * p->n};
        rc = mip_set_instances(t, 2, ro, co, BP_MEM_HOST, s);
        if (rc != BP_OK) {
            mip_free(t);
            return rc;
        }
        p->twin = t;
        p->free_hooks[1] = twin_free;
    }
    *out = p->twin;
    return BP_OK;
}

__global__ void k_pair_of(int npairs, const int* var, int* pair_of) {
    // first pair of each variable wins
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < npairs; i += gridDim.x * blockDim.x)
        atomicMin(&pair_of[var[i]], i);
}

__global__ void k_pair_of_clear(int n, int* pair_of) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x)
        pair_of[j] = pair_of[j] == INT_MAX ? -1 : pair_of[j];
}

__global__ void k_fill_int(int n, int* a, int v) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) a[j] = v;
}

// start bounds of the final check: the caller's bounds with the integer variables at x_out
__global__ void k_fix_ints(int n, const unsigned char* is_int, const double* lb, const double* ub, const double* xo,
                           double* l, double* u) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        l[j] = is_int[j] ? xo[j] : lb[j];
        u[j] = is_int[j] ? xo[j] : ub[j];
    }
}

__global__ void k_finalize(int n, const unsigned char* is_int, const double* x, const double* l, const double* u,
                           int rounding_infeasible, double* x_out) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        if (is_int[j]) {
            double v = l[j];
            if (l[j] < u[j]) v = clampd(floor(__dadd_rn(clampd(x[j], l[j], u[j]), 0.5)), l[j], u[j]);
            x_out[j] = v;
        } else {
            x_out[j] = clampd(x[j], l[j], u[j]);
        }
    }
}

// ------------------------------------------------------------------------ repair
// The repair of Algorithm 1 (Section 2.3): see fix_and_propagate's documentation.  The fixings
// by choice are kept on the device: chosen[j] and its value cval[j].

__global__ void k_mark_chosen(int bsize, const int* bulk, const double* v, unsigned char* chosen, double* cval) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < bsize; i += gridDim.x * blockDim.x) {
        chosen[bulk[i]] = 1;
        cval[bulk[i]] = v[i];
    }
}

// the start of one repair propagation: the caller's bounds with every fixing by choice, and the
// failed variable j at v (entered as a fixing by choice)
// (j = -1 after the first cycle: j is then one of the fixings, possibly moved)
__global__ void k_repair_start(int n, const double* lb, const double* ub, unsigned char* chosen, double* cval, int j,
                               double v, double* fl, double* fu) {
    if (j >= 0 && blockIdx.x == 0 && threadIdx.x == 0) {
        chosen[j] = 1;
        cval[j] = v;
    }
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const bool c = chosen[i] != 0 || i == j;
        const double x = i == j ? v : cval[i];
        fl[i] = c ? x : lb[i];
        fu[i] = c ? x : ub[i];
    }
}

constexpr int kRepThreads = 256;

// the minimal activity of row k under (l, u) over one block: finite part, infinite terms
__device__ void block_min_activity(const DevProblem& P, int k, const double* l, const double* u, double* red,
                                   int* redn, double* minfin, int* ninf) {
    double acc = 0.0;
    int ni = 0;
    for (int q = P.row_ptr[k] + threadIdx.x; q < P.row_ptr[k + 1]; q += kRepThreads) {
        const double a = P.val[q];
        const int j = P.col[q];
        const double b = a > 0 ? l[j] : u[j];
        if (isinf(b)) ++ni;
        else acc = __dadd_rn(acc, __dmul_rn(a, b));
    }
    red[threadIdx.x] = acc;
    redn[threadIdx.x] = ni;
    __syncthreads();
    for (int o = kRepThreads / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            red[threadIdx.x] = __dadd_rn(red[threadIdx.x], red[threadIdx.x + o]);
            redn[threadIdx.x] += redn[threadIdx.x + o];
        }
        __syncthreads();
    }
    *minfin = red[0];
    *ninf = redn[0];
    __syncthreads();
}

// ceil(e / c) for e > 0, c > 0, corrected to the exact integer quotient's ceiling when both are
// integers (their products are exact below 2^53)
__device__ __forceinline__ double ceil_div(double e, double c) {
    double d = ceil(__ddiv_rn(e, c));
    if (e == floor(e) && c == floor(c)) {
        for (int it = 0; it < 4 && d > 1.0 && __dmul_rn(d - 1.0, c) >= e; ++it) d -= 1.0;
        for (int it = 0; it < 4 && __dmul_rn(d, c) < e; ++it) d += 1.0;
    }
    return d;
}

// One repair step after an infeasible propagation (fl, fu: its final bounds; k: its first
// infeasible row or -1; w: its first crossing variable or -1).  The target row is k, else the
// smallest row of w violated under (fl, fu); each fixed variable of it proposes the move that
// makes the row feasible alone, capped by the caller's bounds; the move that lowers the minimal
// activity most (ties: smallest variable) is applied to cval.  *out = 1 when a move was made.
// One block.
__global__ void __launch_bounds__(kRepThreads) k_repair_shift(DevProblem P, const double* fl, const double* fu,
                                                              const double* lb, const double* ub,
                                                              const unsigned char* chosen, double* cval, int k, int w,
                                                              int* out) {
    __shared__ double red[kRepThreads];
    __shared__ int redn[kRepThreads];
    __shared__ int red_i[kRepThreads];
    int target = k;
    if (target < 0 && w >= 0) {
        int best = INT_MAX;
        for (int s = P.col_ptr[w]; s < P.col_ptr[w + 1]; ++s) {
            const int kk = P.row_idx[s];
            double mf;
            int ni;
            block_min_activity(P, kk, fl, fu, red, redn, &mf, &ni);
            const double2 g2 = P.grow[kk];
            if (ni == 0 && isfinite(g2.x) && mf > g2.y && kk < best) best = kk;
        }
        target = best == INT_MAX ? -1 : best;
    }
    if (target < 0) {
        if (threadIdx.x == 0) *out = 0;
        return;
    }
    double mf;
    int ni;
    block_min_activity(P, target, fl, fu, red, redn, &mf, &ni);
    const double e = __dsub_rn(mf, P.grow[target].x);
    if (ni != 0 || !(e > 0.0)) {
        if (threadIdx.x == 0) *out = 0;
        return;
    }
    // each thread's best move over its nonzeros, then a block reduction (largest reduction,
    // smallest variable)
    double br = 0.0;
    int bi = INT_MAX;
    for (int q = P.row_ptr[target] + threadIdx.x; q < P.row_ptr[target + 1]; q += kRepThreads) {
        const int i = P.col[q];
        if (!chosen[i]) continue;
        const double a = P.val[q], aa = fabs(a);
        const double need = ceil_div(e, aa);
        const double room = a > 0 ? floor(__dsub_rn(cval[i], lb[i])) : floor(__dsub_rn(ub[i], cval[i]));
        const double d = need < room ? need : room;
        if (!(d > 0.0)) continue;
        const double rr = __dmul_rn(aa, d);
        if (rr > br || (rr == br && i < bi)) {
            br = rr;
            bi = i;
        }
    }
    red[threadIdx.x] = br;
    red_i[threadIdx.x] = bi;
    __syncthreads();
    for (int o = kRepThreads / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            const double r2 = red[threadIdx.x + o];
            const int i2 = red_i[threadIdx.x + o];
            if (r2 > red[threadIdx.x] || (r2 == red[threadIdx.x] && i2 < red_i[threadIdx.x])) {
                red[threadIdx.x] = r2;
                red_i[threadIdx.x] = i2;
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const int i = red_i[0];
        if (i == INT_MAX) {
            *out = 0;
            return;
        }
        // the chosen move again (its coefficient from the row)
        double a = 0.0;
        for (int q = P.row_ptr[target]; q < P.row_ptr[target + 1]; ++q)
            if (P.col[q] == i) a = P.val[q];
        const double aa = fabs(a);
        const double room = a > 0 ? floor(__dsub_rn(cval[i], lb[i])) : floor(__dsub_rn(ub[i], cval[i]));
        const double need = ceil_div(e, aa);
        const double d = need < room ? need : room;
        cval[i] = a > 0 ? __dsub_rn(cval[i], d) : __dadd_rn(cval[i], d);
        *out = 1;
    }
}

static int gridn(long long work) {
    long long b = (work + 255) / 256;
    return (int)(b < 1 ? 1 : (b > 1216 ? 1216 : b));
}

// per-bulk control words read back by the host
struct FpCtl {
    int kept[2];
    int ucnt[2];      // unfixed integer variables under each candidate's propagated bounds
    bp_result res[2];
    FpSingleOut single;   // counters of a device-driven run of one-variable bulks
    int rep_j;            // repair: the failed variable and its drawn value, read back
    double rep_v;
    int rep_moved;        // repair: a fixing was moved
};

// The current bounds as ordered keys (cur) and in both copies of both key buffers of the
// instance pair: the state the device-driven one-variable bulks start from.
__global__ void k_keys_init(int n, const unsigned char* is_int, const double* l, const double* u, longlong2* cur,
                            longlong2* bk0, longlong2* bk1) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        const longlong2 k = normalized_keys(l[j], u[j], is_int[j] != 0);
        cur[j] = k;
        bk0[j] = k;
        bk0[(size_t)n + j] = k;
        bk1[j] = k;
        bk1[(size_t)n + j] = k;
    }
}

__global__ void k_keys_out(int n, const longlong2* cur, double* l, double* u) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        const longlong2 k = cur[j];
        l[j] = kdec(k.x);
        u[j] = kdec(k.y);
    }
}

// Blocks of row c (blockIdx.y) count the integer variables left unfixed by candidate c (bounds
// l + c n, u + c n) into out[c], zeroed by k_fill_pair: the next bulk's unfixed count, read with
// the candidates' results in one transfer.
__global__ void k_count_unset2(int nint, const int* order, const double* l, const double* u, int n, int* out) {
    __shared__ int part[8];
    const double* lc = l + (size_t)blockIdx.y * n;
    const double* uc = u + (size_t)blockIdx.y * n;
    int c = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nint; i += gridDim.x * blockDim.x) {
        const int j = order[i];
        c += lc[j] < uc[j] ? 1 : 0;
    }
    for (int off = 16; off > 0; off >>= 1) c += __shfl_xor_sync(0xffffffffu, c, off);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        int t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += part[w];
        if (t) atomicAdd(out + blockIdx.y, t);
    }
}

// both candidates start from the current bounds: (l, u) into both halves of (cl, cu)
__global__ void k_fill_pair(int n, const double* l, const double* u, double* cl, double* cu, int* ucnt) {
    if (blockIdx.x == 0 && threadIdx.x < 2) ucnt[threadIdx.x] = 0;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        const double a = l[j], b = u[j];
        cl[j] = a;
        cl[n + j] = a;
        cu[j] = b;
        cu[n + j] = b;
    }
}

}  // namespace gpubp

using namespace gpubp;

extern "C" void fp_params_default(fp_params* p) {
    if (!p) return;
    p->seed = 1;
    p->bulk_rule = FP_BULK_SQRT;
    p->last_single = 36;
    p->fraction = 0.01;
    p->theta = 1e-3;
    p->max_rounds = 10000;
    p->repair_max = 0;
    p->repair_cycles = 8;
    p->reserved = 0;
    p->order_score = nullptr;
    p->up_prob = nullptr;
}

extern "C" int fix_and_propagate(mip_problem* p, const double* x, const double* lb, const double* ub,
                                 const fp_cache* cache, const fp_params* params, double* x_out, fp_result* result,
                                 void* stream) {
    if (!p || !result || (p->n && (!x || !lb || !ub || !x_out))) {
        set_error("fix_and_propagate: null argument");
        return BP_ERR_INVALID;
    }
    fp_params prm;
    if (params) prm = *params;
    else fp_params_default(&prm);
    if (!(prm.theta >= 0.0) || prm.max_rounds < 0 || prm.last_single < 0 ||
        (prm.bulk_rule != FP_BULK_SQRT && prm.bulk_rule != FP_BULK_FRACTION) ||
        (prm.bulk_rule == FP_BULK_FRACTION && !(prm.fraction > 0.0))) {
        set_error("fix_and_propagate: invalid parameters");
        return BP_ERR_INVALID;
    }
    if (cache && cache->npairs > 0 &&
        (!cache->var || !cache->boxes || !cache->status || !cache->offsets)) {
        set_error("fix_and_propagate: incomplete cache");
        return BP_ERR_INVALID;
    }
    if (prm.repair_max < 0 || (prm.repair_max > 0 && prm.repair_cycles < 1)) {
        set_error("fix_and_propagate: invalid repair parameters");
        return BP_ERR_INVALID;
    }
    if (prm.repair_max > 0 && cache && cache->npairs > 0) {
        set_error("fix_and_propagate: the repair is defined without a probing cache");
        return BP_ERR_INVALID;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const int n = p->n;
    memset(result, 0, sizeof(*result));
    // scratch (stream-ordered allocations, freed at the end)
    std::vector<void*> tmp;
    auto alloc = [&](auto** ptr, size_t count) -> int {
        void* q = nullptr;
        cudaError_t e = cudaMallocAsync(&q, (count ? count : 1) * sizeof(**ptr), s);
        if (e != cudaSuccess) return fail_cuda(e, "cudaMallocAsync");
        tmp.push_back(q);
        *ptr = static_cast<std::remove_reference_t<decltype(*ptr)>>(q);
        return BP_OK;
    };
    auto release = [&]() {
        for (void* q : tmp) cudaFreeAsync(q, s);
        tmp.clear();
    };
    int rc = BP_OK;
    double *Bl, *Bu, *cl[2], *cu[2], *v[2], *rmin, *L4, *U4;
    int *flag, *pos, *ivars, *order, *work, *twork, *rninf, *dlist, *dcnt, *pair_of = nullptr, *total;
    unsigned long long *keys, *tkeys;
    unsigned char* chosen = nullptr;   // repair: fixings by choice and their values
    double* cval = nullptr;
    int* rep_out = nullptr;
    longlong2* curk = nullptr;     // device-driven one-variable bulks (allocated on first use)
    int *vdirty = nullptr, *dirtyl = nullptr, *words = nullptr;
    FpSingleOut* sout = nullptr;
    FpCtl* dctl;
    FpCtl* hctl = nullptr;
#define FP_ALLOC(ptr, cnt)                      \
    do {                                        \
        rc = alloc(&ptr, (size_t)(cnt));        \
        if (rc != BP_OK) { release(); return rc; } \
    } while (0)
    // Four bound slots: the current bounds in one, the two candidates in the two halves of the
    // other pair (slots 0-1 or 2-3), so the instance pair reads them as one array and a picked
    // candidate becomes the current bounds without a copy.
    FP_ALLOC(L4, 4 * (size_t)n);
    FP_ALLOC(U4, 4 * (size_t)n);
    int cur = 0;
    Bl = L4;
    Bu = U4;
    for (int c = 0; c < 2; ++c) FP_ALLOC(v[c], n);
    FP_ALLOC(dlist, 2 * (size_t)n);
    FP_ALLOC(rmin, p->m);
    FP_ALLOC(rninf, p->m);
    FP_ALLOC(flag, n);
    FP_ALLOC(pos, n);
    FP_ALLOC(ivars, n);
    FP_ALLOC(order, n);
    FP_ALLOC(work, n);
    FP_ALLOC(twork, n);
    FP_ALLOC(keys, n);
    FP_ALLOC(tkeys, n);
    FP_ALLOC(dcnt, 2);
    FP_ALLOC(total, 1);
    FP_ALLOC(dctl, 1);
    if (cudaMallocHost(&hctl, sizeof(FpCtl)) != cudaSuccess) {
        release();
        set_error("pinned host allocation failed");
        return BP_ERR_OOM;
    }
    auto fail = [&](int code) {
        release();
        cudaFreeHost(hctl);
        return code;
    };
#define FP_TRY(expr)                      \
    do {                                  \
        int _r = (expr);                  \
        if (_r != BP_OK) return fail(_r); \
    } while (0)
#define FP_CUDA(expr)                                        \
    do {                                                     \
        cudaError_t _e = (expr);                             \
        if (_e != cudaSuccess) return fail(fail_cuda(_e, #expr)); \
    } while (0)
    const bool use_cache = cache && cache->npairs > 0;
    const bool repair_on = prm.repair_max > 0;
    int repairs_tried = 0;
    if (repair_on) {
        FP_TRY(alloc(&chosen, (size_t)n));
        FP_TRY(alloc(&cval, (size_t)n));
        FP_TRY(alloc(&rep_out, 1));
        FP_CUDA(cudaMemsetAsync(chosen, 0, (size_t)(n ? n : 1), s));
    }
    if (use_cache) {
        FP_ALLOC(pair_of, n);
        k_fill_int<<<gridn(n), 256, 0, s>>>(n, pair_of, INT_MAX);
        k_pair_of<<<gridn(cache->npairs), 256, 0, s>>>(cache->npairs, cache->var, pair_of);
        k_pair_of_clear<<<gridn(n), 256, 0, s>>>(n, pair_of);
    }
    mip_problem* tw = nullptr;
    FP_TRY(twin_problem(p, s, &tw));
    // ---- propagate the start bounds
    FP_CUDA(cudaMemcpyAsync(Bl, lb, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    FP_CUDA(cudaMemcpyAsync(Bu, ub, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    FP_TRY(launch_propagate(p, Bl, Bu, nullptr, 0, prm.theta, prm.max_rounds, nullptr, s));
    FP_CUDA(cudaMemcpyAsync(hctl->res, p->w.dres, sizeof(bp_result), cudaMemcpyDeviceToHost, s));
    // integer variables and their initial order
    k_intvars_flag<<<gridn(n), 256, 0, s>>>(n, p->dp.is_int, flag);
    FP_TRY(scan_exclusive(flag, pos, n, total, s));
    k_compact_idx<<<gridn(n), 256, 0, s>>>(n, flag, pos, ivars);
    int nint = 0;
    FP_CUDA(cudaMemcpyAsync(&nint, total, sizeof(int), cudaMemcpyDeviceToHost, s));
    FP_CUDA(cudaStreamSynchronize(s));
    if (hctl->res[0].error) return fail(BP_ERR_TIMEOUT);
    result->bp_runs = 1;
    result->nnz_updates = hctl->res[0].nnz_updates;
    bool rounding_infeasible = hctl->res[0].status == BP_INFEASIBLE;
    FP_CUDA(cudaMemcpyAsync(order, ivars, sizeof(int) * nint, cudaMemcpyDeviceToDevice, s));
    {
        const int passes[3] = {0, 1, 2};
        for (int which : passes) {
            if (which == 1 && !prm.order_score) continue;
            if (nint == 0) break;
            k_initial_keys<<<gridn(nint), 256, 0, s>>>(nint, order, x, Bl, Bu, prm.order_score, which, keys);
            FP_TRY(radix_sort_pairs(keys, order, tkeys, twork, nint, 0, which == 2 ? 8 : 64, s));
        }
    }
    // Repair of a one-variable bulk that failed both ways (variable j, drawn value v0): returns 1
    // when a propagation became feasible (its bounds are then the current ones), 0 when not,
    // or minus an error code.
    auto do_repair = [&](int j, double v0) -> int {
        const int fs = (cur + 2) % 4;
        double* fl = L4 + (size_t)fs * n;
        double* fu = U4 + (size_t)fs * n;
        for (int c = 0; c < prm.repair_cycles; ++c) {
            k_repair_start<<<gridn(n), 256, 0, s>>>(n, lb, ub, chosen, cval, c == 0 ? j : -1, v0, fl, fu);
            if (cudaGetLastError() != cudaSuccess) return -BP_ERR_CUDA;
            int rc2 = launch_propagate(p, fl, fu, nullptr, 0, prm.theta, prm.max_rounds, nullptr, s);
            if (rc2 != BP_OK) return -rc2;
            if (cudaMemcpyAsync(&hctl->res[0], p->w.dres, sizeof(bp_result), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                cudaStreamSynchronize(s) != cudaSuccess)
                return -BP_ERR_CUDA;
            const bp_result r = hctl->res[0];
            if (r.error) return -BP_ERR_TIMEOUT;
            result->bp_runs++;
            result->repair_runs++;
            result->nnz_updates += r.nnz_updates;
            if (r.status != BP_INFEASIBLE) {
                cur = fs;
                Bl = fl;
                Bu = fu;
                return 1;
            }
            k_repair_shift<<<1, kRepThreads, 0, s>>>(p->dp, fl, fu, lb, ub, chosen, cval, r.first_infeasible_row,
                                                      r.first_infeasible_var, rep_out);
            if (cudaGetLastError() != cudaSuccess) return -BP_ERR_CUDA;
            if (cudaMemcpyAsync(&hctl->rep_moved, rep_out, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                cudaStreamSynchronize(s) != cudaSuccess)
                return -BP_ERR_CUDA;
            if (!hctl->rep_moved) return 0;
        }
        return 0;
    };
    std::vector<int> recq;
    size_t rec_pos = 0;
    unsigned long long bulk_index = 0;
    bool have_nun = false;   // the unfixed count came with the previous bulk's results
    int next_nun = 0;
    while (!rounding_infeasible) {
        // unfixed integer variables in the initial order
        int nun = 0;
        if (nint) {
            k_unset_flag<<<gridn(nint), 256, 0, s>>>(nint, order, Bl, Bu, flag);
            FP_TRY(scan_exclusive(flag, pos, nint, total, s));
            k_compact_list<<<gridn(nint), 256, 0, s>>>(nint, order, flag, pos, work);
            if (have_nun) {
                nun = next_nun;
            } else {
                FP_CUDA(cudaMemcpyAsync(&nun, total, sizeof(int), cudaMemcpyDeviceToHost, s));
                FP_CUDA(cudaStreamSynchronize(s));
            }
        }
        have_nun = false;
        if (nun == 0) break;
        long long bsize = 1;
        bool single = false;
        const int* bulk = work;
        // recovery: the failed bulk's variables one at a time, skipping those fixed meanwhile
        while (rec_pos < recq.size()) {
            double lu[2];
            FP_CUDA(cudaMemcpyAsync(&lu[0], Bl + recq[rec_pos], sizeof(double), cudaMemcpyDeviceToHost, s));
            FP_CUDA(cudaMemcpyAsync(&lu[1], Bu + recq[rec_pos], sizeof(double), cudaMemcpyDeviceToHost, s));
            FP_CUDA(cudaStreamSynchronize(s));
            if (lu[0] < lu[1]) break;
            ++rec_pos;
        }
        if (rec_pos < recq.size()) {
            const int j = recq[rec_pos++];
            FP_CUDA(cudaMemcpyAsync(twork, &j, sizeof(int), cudaMemcpyHostToDevice, s));
            bulk = twork;
            bsize = 1;
            single = true;
        } else {
            recq.clear();
            rec_pos = 0;
            if (nun <= prm.last_single) {
                bsize = 1;
            } else if (prm.bulk_rule == FP_BULK_SQRT) {
                long long r = (long long)std::sqrt((double)nun);
                while (r * r > nun) --r;
                while ((r + 1) * (r + 1) <= nun) ++r;
                bsize = r * r == nun ? r : r + 1;
            } else {
                bsize = (long long)std::ceil(prm.fraction * (double)nint);
                if (bsize < 1) bsize = 1;
            }
            if (bsize > nun) bsize = nun;
            // a learned order score replaces the per-bulk implied-slack order
            if (bsize > 1 && !prm.order_score) {
                if (p->m) k_row_act<<<gridn((long long)p->m * 32), 256, 0, s>>>(p->dp, Bl, Bu, rmin, rninf);
                k_implied_slack<<<gridn(nun), 256, 0, s>>>(p->dp, nun, work, rmin, rninf, keys);
                if (bsize <= kSelectMax) {
                    // only the bulk is needed: the first bsize of the stable sort, selected
                    FP_TRY(select_smallest(keys, work, nun, (int)bsize, twork, s));
                    bulk = twork;
                } else {
                    FP_TRY(radix_sort_pairs(keys, work, tkeys, twork, nun, 0, 64, s));
                }
            }
            single = bsize == 1;
        }
        // candidate values and start boxes of the two vectors
        k_draws<<<gridn(bsize), 256, 0, s>>>((int)bsize, bulk, x, Bl, Bu, prm.seed, bulk_index, single ? 1 : 0,
                                               prm.up_prob, v[0], v[1]);
        FP_CUDA(cudaMemsetAsync(dcnt, 0, sizeof(int), s));
        const int cp = ((cur >> 1) ^ 1) * 2;   // first slot of the candidates' pair
        cl[0] = L4 + (size_t)cp * n;
        cu[0] = U4 + (size_t)cp * n;
        cl[1] = cl[0] + n;
        cu[1] = cu[0] + n;
        k_fill_pair<<<gridn(n), 256, 0, s>>>(n, Bl, Bu, cl[0], cu[0], dctl->ucnt);
        for (int c = 0; c < 2; ++c) {
            if (use_cache) {
                k_apply_cache<<<1, 32, 0, s>>>((int)bsize, bulk, v[c], cl[c], cu[c], p->dp.is_int, pair_of, *cache,
                                               &dctl->kept[c]);
            } else {
                k_apply_plain<<<gridn(bsize), 256, 0, s>>>((int)bsize, bulk, v[c], cl[c], cu[c], &dctl->kept[c]);
            }
            k_diff<<<gridn(n), 256, 0, s>>>(n, cl[c], cu[c], Bl, Bu, c * n, dlist, dcnt);
            FP_CUDA(cudaGetLastError());
        }
        // double propagation in one launch: each vector from the rows of the variables it
        // changes, as the two instances of the pair
        FP_TRY(launch_propagate(tw, cl[0], cu[0], nullptr, 0, prm.theta, prm.max_rounds, nullptr, s, dlist, dcnt, 2,
                                tw->inst_row_off, tw->inst_col_off));
        FP_CUDA(cudaMemcpyAsync(dctl->res, tw->w.dres, 2 * sizeof(bp_result), cudaMemcpyDeviceToDevice, s));
        {
            const int gx = (nint + 1023) / 1024 < 64 ? (nint + 1023) / 1024 : 64;
            k_count_unset2<<<dim3(gx > 0 ? gx : 1, 2), 256, 0, s>>>(nint, order, cl[0], cu[0], n, dctl->ucnt);
        }
        FP_CUDA(cudaMemcpyAsync(hctl, dctl, sizeof(FpCtl), cudaMemcpyDeviceToHost, s));
        FP_CUDA(cudaStreamSynchronize(s));
        bool feas[2];
        for (int c = 0; c < 2; ++c) {
            if (hctl->res[c].error) return fail(BP_ERR_TIMEOUT);
            if (hctl->kept[c] > 0) {
                result->bp_runs++;
                result->nnz_updates += hctl->res[c].nnz_updates;
            }
            feas[c] = hctl->kept[c] > 0 && hctl->res[c].status != BP_INFEASIBLE;
        }
        result->bulks++;
        bulk_index++;
        const int pick = feas[0] ? 0 : (feas[1] ? 1 : -1);
        if (pick >= 0) {
            result->fixed_by_choice += hctl->kept[pick];
            cur = cp + pick;
            Bl = L4 + (size_t)cur * n;
            Bu = U4 + (size_t)cur * n;
            next_nun = hctl->ucnt[pick];
            have_nun = nint > 0;
            if (repair_on) {
                k_mark_chosen<<<gridn(bsize), 256, 0, s>>>((int)bsize, bulk, v[pick], chosen, cval);
                FP_CUDA(cudaGetLastError());
            }
        } else if (!single && !use_cache) {
            // recovery on the device: the failed bulk's variables one at a time, in one launch
            result->recoveries++;
            if (!curk) {
                FP_TRY(alloc(&curk, (size_t)n));
                FP_TRY(alloc(&vdirty, 2 * (size_t)n));
                FP_TRY(alloc(&dirtyl, 2 * (size_t)n));
                FP_TRY(alloc(&words, 4));
                FP_TRY(alloc(&sout, 1));
            }
            // the queue from qstart; after a successful repair the launch resumes behind the
            // repaired variable
            for (int qstart = 0; qstart < (int)bsize;) {
                // cleared for every run: a plain propagation launch in between may have restarted
                // the stamps, which this array's entries are compared with
                FP_CUDA(cudaMemsetAsync(vdirty, 0, sizeof(int) * 2 * (size_t)n, s));
                k_keys_init<<<gridn(n), 256, 0, s>>>(n, p->dp.is_int, Bl, Bu, curk, tw->w.bkey[0], tw->w.bkey[1]);
                FP_CUDA(cudaGetLastError());
                FP_TRY(launch_fp_single(tw, n, curk, bulk + qstart, (int)bsize - qstart, x, prm.up_prob, prm.seed,
                                        bulk_index, prm.theta, prm.max_rounds, vdirty, dirtyl, words, sout, chosen,
                                        cval, s));
                k_keys_out<<<gridn(n), 256, 0, s>>>(n, curk, Bl, Bu);
                FP_CUDA(cudaGetLastError());
                FP_CUDA(cudaMemcpyAsync(&hctl->single, sout, sizeof(FpSingleOut), cudaMemcpyDeviceToHost, s));
                FP_CUDA(cudaStreamSynchronize(s));
                const FpSingleOut so = hctl->single;
                if (so.error) return fail(so.error);
                result->bulks += so.bulks;
                bulk_index += (unsigned long long)so.bulks;
                result->bp_runs += so.bp_runs;
                result->nnz_updates += so.nnz_updates;
                result->fixed_by_choice += so.fixed;
                if (!so.infeasible) break;
                if (!(repair_on && repairs_tried < prm.repair_max)) {
                    rounding_infeasible = true;
                    break;
                }
                repairs_tried++;
                const int rr = do_repair(so.j, so.v0);
                if (rr < 0) return fail(-rr);
                if (!rr) {
                    rounding_infeasible = true;
                    break;
                }
                result->repairs++;
                qstart += so.stop_q + 1;
            }
            have_nun = false;
        } else if (!single) {
            recq.resize((size_t)bsize);
            FP_CUDA(cudaMemcpyAsync(recq.data(), bulk, sizeof(int) * bsize, cudaMemcpyDeviceToHost, s));
            FP_CUDA(cudaStreamSynchronize(s));
            rec_pos = 0;
            result->recoveries++;
            next_nun = nun;   // the bounds did not move
            have_nun = true;
        } else if (repair_on && repairs_tried < prm.repair_max) {
            // a one-variable bulk failed both ways: repair
            repairs_tried++;
            FP_CUDA(cudaMemcpyAsync(&hctl->rep_j, bulk, sizeof(int), cudaMemcpyDeviceToHost, s));
            FP_CUDA(cudaMemcpyAsync(&hctl->rep_v, v[0], sizeof(double), cudaMemcpyDeviceToHost, s));
            FP_CUDA(cudaStreamSynchronize(s));
            const int rr = do_repair(hctl->rep_j, hctl->rep_v);
            if (rr < 0) return fail(-rr);
            if (rr) result->repairs++;
            else rounding_infeasible = true;
            have_nun = false;
        } else {
            rounding_infeasible = true;
        }
    }
    k_finalize<<<gridn(n), 256, 0, s>>>(n, p->dp.is_int, x, Bl, Bu, rounding_infeasible ? 1 : 0, x_out);
    FP_CUDA(cudaGetLastError());
    // final check: one propagation of the caller's bounds with every integer variable fixed at
    // its value (in a slot of the pair that does not hold the current bounds)
    if (!rounding_infeasible) {
        const int fs = (cur + 2) % 4;
        double* fl = L4 + (size_t)fs * n;
        double* fu = U4 + (size_t)fs * n;
        k_fix_ints<<<gridn(n), 256, 0, s>>>(n, p->dp.is_int, lb, ub, x_out, fl, fu);
        FP_CUDA(cudaGetLastError());
        FP_TRY(launch_propagate(p, fl, fu, nullptr, 0, prm.theta, prm.max_rounds, nullptr, s));
        FP_CUDA(cudaMemcpyAsync(&hctl->res[0], p->w.dres, sizeof(bp_result), cudaMemcpyDeviceToHost, s));
        FP_CUDA(cudaStreamSynchronize(s));
        if (hctl->res[0].error) return fail(BP_ERR_TIMEOUT);
        result->refuted = hctl->res[0].status == BP_INFEASIBLE ? 1 : 0;
    }
    result->status = (rounding_infeasible || result->refuted) ? FP_INFEASIBLE : FP_FEASIBLE;
    release();
    FP_CUDA(cudaStreamSynchronize(s));
    cudaFreeHost(hctl);
    p->last_stream = s;
    return BP_OK;
}
