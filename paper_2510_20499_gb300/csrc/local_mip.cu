// The local search's move scoring (Section 2.4, the paper's GPU Local-MIP): the mixed-tight-move
// core under a weighted violation F = sum_k w_k max(0, (A x)_k - g_k).
//
// Per iteration, every candidate and its full score are recomputed (as the paper does, instead
// of the score deltas of the original Feasibility Jump):
//   k_ls_score   a warp per violated row: each lane takes nonzeros of the row, forms the value
//                that alone satisfies the row (integers by the smallest integer step, clamped to
//                the bounds) and scores it by walking the variable's column (rows ascending);
//                warp and block reductions keep the best (largest score; ties: smallest variable,
//                then smallest value), one per block;
//   k_ls_apply   one block: the best over the blocks (a total order, so the result does not
//                depend on the reduction's order); a positive score moves the variable and
//                updates the activities of its column, otherwise the weights are to grow;
//   k_ls_bump    every violated row's weight grows by 1 when no move improved.
// Everything stays on the device (no host read per iteration).  The activities start from a
// thread-per-row sum in row order and are updated in the order of the moves, so the search is
// bit-for-bit that of a sequential implementation with the same operation order.
#include <climits>
#include <cmath>

#include "bp_host.h"

namespace gpubp {

constexpr int kLsThreads = 256;
constexpr int kLsRedBlocks = 304;

struct LsKey {
    double score;
    double t;
    int j;
    int pad;
};

__device__ __forceinline__ LsKey ls_none() { return LsKey{-INFINITY, INFINITY, INT_MAX, 0}; }

// a before b: larger score; ties: smaller variable, then smaller value
__device__ __forceinline__ bool ls_before(const LsKey& a, const LsKey& b) {
    if (a.score != b.score) return a.score > b.score;
    if (a.j != b.j) return a.j < b.j;
    return a.t < b.t;
}

__device__ __forceinline__ LsKey ls_shfl(const LsKey& k, int lane) {
    LsKey o;
    o.score = __shfl_sync(0xffffffffu, k.score, lane);
    o.t = __shfl_sync(0xffffffffu, k.t, lane);
    o.j = __shfl_sync(0xffffffffu, k.j, lane);
    o.pad = 0;
    return o;
}

struct LsCtl {
    int nviol;        // violated rows seen by this iteration's scoring pass
    int bump;         // the weights grow in this iteration
    int moves, bumps;
};

__global__ void k_ls_activities(DevProblem P, const double* __restrict__ x, double* __restrict__ L) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < P.m; k += gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int q = P.row_ptr[k]; q < P.row_ptr[k + 1]; ++q) s = __dadd_rn(s, __dmul_rn(P.val[q], x[P.col[q]]));
        L[k] = s;
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

__global__ void __launch_bounds__(kLsThreads) k_ls_score(DevProblem P, const double* __restrict__ lb,
                                                         const double* __restrict__ ub, const double* __restrict__ x,
                                                         const double* __restrict__ w, const double* __restrict__ L,
                                                         LsKey* __restrict__ part, LsCtl* ctl) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
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
            double t;
            if (P.is_int[j]) {
                const double d = ls_ceil_div(v, fabs(a));
                t = a > 0.0 ? __dsub_rn(xj, d) : __dadd_rn(xj, d);
            } else {
                t = __dsub_rn(xj, __ddiv_rn(v, a));
            }
            t = t < lb[j] ? lb[j] : t;   // max(t, l), then min(., u)
            t = t > ub[j] ? ub[j] : t;
            if (t == xj) continue;
            const double dx = __dsub_rn(t, xj);
            double s = 0.0;
            // the column's rows in order; the loads of four entries are issued together
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
                    ll[i] = L[r];
                    ww[i] = w[r];
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
            const LsKey key{s, t, j, 0};
            if (ls_before(key, best)) best = key;
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

__global__ void __launch_bounds__(kLsThreads) k_ls_apply(DevProblem P, double* __restrict__ x, double* __restrict__ L,
                                                         const LsKey* __restrict__ part, int nparts, LsCtl* ctl) {
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
    const int nviol = ctl->nviol;
    __syncthreads();
    if (best.j != INT_MAX && best.score > 0.0) {
        const int j = best.j;
        const double dx = __dsub_rn(best.t, x[j]);
        for (int c = P.col_ptr[j] + threadIdx.x; c < P.col_ptr[j + 1]; c += kLsThreads) {
            const int r = P.row_idx[c];
            L[r] = __dadd_rn(L[r], __dmul_rn(P.col_val[c], dx));
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            x[j] = best.t;
            ctl->moves += 1;
            ctl->bump = 0;
        }
    } else if (threadIdx.x == 0) {
        ctl->bump = nviol > 0 ? 1 : 0;
        if (nviol > 0) ctl->bumps += 1;
    }
    if (threadIdx.x == 0) ctl->nviol = 0;
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

extern "C" int local_search_mtm(mip_problem* p, const double* lb, const double* ub, double* x, double* w,
                                const ls_params* params, ls_result* result, void* stream) {
    if (!p || !params || !result || (p->n && (!lb || !ub || !x)) || (p->m && !w)) {
        set_error("local_search_mtm: null argument");
        return BP_ERR_INVALID;
    }
    if (params->iterations < 0) {
        set_error("local_search_mtm: negative iteration count");
        return BP_ERR_INVALID;
    }
    cudaStream_t s = (cudaStream_t)stream;
    memset(result, 0, sizeof(*result));
    void *pL = nullptr, *pPart = nullptr, *pCtl = nullptr, *pSum = nullptr, *pOut = nullptr;
    // the scoring pass on every resident block (its per-block bests are reduced by k_ls_apply)
    static int occ_score = -1;
    if (occ_score < 0) {
        cudaError_t oe = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_score, k_ls_score, kLsThreads, 0);
        if (oe != cudaSuccess) return fail_cuda(oe, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
    }
    const int grid_score = p->sms * (occ_score > 0 ? occ_score : 1);
    auto release = [&]() {
        for (void* q : {pL, pPart, pCtl, pSum, pOut})
            if (q) cudaFreeAsync(q, s);
    };
    cudaError_t e = cudaSuccess;
    if ((e = cudaMallocAsync(&pL, sizeof(double) * (size_t)(p->m ? p->m : 1), s)) != cudaSuccess ||
        (e = cudaMallocAsync(&pPart, sizeof(LsKey) * (size_t)grid_score, s)) != cudaSuccess ||
        (e = cudaMallocAsync(&pCtl, sizeof(LsCtl), s)) != cudaSuccess ||
        (e = cudaMallocAsync(&pSum, sizeof(double) * 3 * kLsRedBlocks, s)) != cudaSuccess ||
        (e = cudaMallocAsync(&pOut, sizeof(double) * 3, s)) != cudaSuccess) {
        release();
        return fail_cuda(e, "cudaMallocAsync");
    }
    double* L = static_cast<double*>(pL);
    LsKey* part = static_cast<LsKey*>(pPart);
    LsCtl* ctl = static_cast<LsCtl*>(pCtl);
    const int grid_rows = p->sms * 8;
    if ((e = cudaMemsetAsync(ctl, 0, sizeof(LsCtl), s)) != cudaSuccess) {
        release();
        return fail_cuda(e, "cudaMemsetAsync");
    }
    k_ls_activities<<<grid_rows, kLsThreads, 0, s>>>(p->dp, x, L);
    for (int it = 0; it < params->iterations; ++it) {
        k_ls_score<<<grid_score, kLsThreads, 0, s>>>(p->dp, lb, ub, x, w, L, part, ctl);
        k_ls_apply<<<1, kLsThreads, 0, s>>>(p->dp, x, L, part, grid_score, ctl);
        k_ls_bump<<<grid_rows, kLsThreads, 0, s>>>(p->dp, L, w, ctl);
    }
    k_ls_summary<<<kLsRedBlocks, kLsThreads, 0, s>>>(p->dp, p->obj, x, w, L, static_cast<double*>(pSum));
    k_ls_summary_finish<<<1, 32, 0, s>>>(static_cast<double*>(pSum), kLsRedBlocks, static_cast<double*>(pOut));
    if ((e = cudaGetLastError()) != cudaSuccess) {
        release();
        return fail_cuda(e, "local search launch");
    }
    double out[3];
    LsCtl hc;
    e = cudaMemcpyAsync(out, pOut, sizeof(out), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hc, ctl, sizeof(hc), cudaMemcpyDeviceToHost, s);
    release();
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail_cuda(e, "local search results");
    result->iterations = params->iterations;
    result->moves = hc.moves;
    result->bumps = hc.bumps;
    result->violated = (int32_t)out[0];
    result->weighted_violation = out[1];
    result->objective = out[2];
    p->last_stream = s;
    return BP_OK;
}
