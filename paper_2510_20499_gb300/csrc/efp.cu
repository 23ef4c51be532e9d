// The extended feasibility pump's orchestration (Section 2.5, Algorithm 2, generation mode):
// extended_fp.  It drives the library's own steps in Algorithm 2's order: the approximate LP
// (pdhg_solve), the rounding (fix_and_propagate), the local search (local_search_mtm); the
// small steps between them are kernels here:
//   k_efp_clip_zero   the all-zero point clamped to the bounds;
//   k_efp_snap        a projection to the nearest multiple of 2^-20, clamped to the bounds (so
//                     that distances are exact sums and the rounding sees the same values as any
//                     implementation of the same steps);
//   k_efp_objective   the projection's objective: +1 for an integer variable at its lower bound,
//                     -1 at its upper bound, 0 otherwise;
//   k_efp_nearest     the nearest integers (ties up), clamped to the bounds;
//   k_efp_distance    sum over integer variables of |a - b| (exact: multiples of 2^-20).
// Improvement mode adds the objective cut c x <= c x* - delta as row m of a second handle,
// assembled on the device (the CSR copied, the nonzero costs compacted by a scan into the new
// row) and loaded again with each incumbent's right-hand side (k_efp_cut_rhs: c x* summed in
// index order by one thread, so the cut is the same as any sequential implementation's).
// The host keeps the round loop and its cycle test (one read of the distance per round).
#include <cmath>
#include <vector>

#include "bp_host.h"

namespace gpubp {

constexpr int kEfpThreads = 256;
constexpr int kEfpBlocks = 304;
constexpr double kSnap = 1048576.0;   // 2^20

__global__ void k_efp_clip_zero(int n, const double* lb, const double* ub, double* x) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        double v = 0.0;
        v = v < lb[j] ? lb[j] : v;
        v = v > ub[j] ? ub[j] : v;
        x[j] = v;
    }
}

__global__ void k_efp_snap(int n, const double* x, const double* lb, const double* ub, double* out) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        double v = __dmul_rn(rint(__dmul_rn(x[j], kSnap)), 1.0 / kSnap);
        v = v < lb[j] ? lb[j] : v;
        v = v > ub[j] ? ub[j] : v;
        out[j] = v;
    }
}

__global__ void k_efp_objective(int n, const unsigned char* is_int, const double* s, const double* lb,
                                const double* ub, double* c) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        double v = 0.0;
        if (is_int[j] && lb[j] < ub[j]) {
            if (s[j] <= lb[j]) v = 1.0;
            else if (s[j] >= ub[j]) v = -1.0;
        }
        c[j] = v;
    }
}

__global__ void k_efp_nearest(int n, const unsigned char* is_int, const double* x, const double* lb, const double* ub,
                              double* out) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        double v = x[j];
        if (is_int[j]) {
            v = floor(__dadd_rn(v, 0.5));
            v = v < lb[j] ? lb[j] : v;
            v = v > ub[j] ? ub[j] : v;
        }
        out[j] = v;
    }
}

__global__ void __launch_bounds__(kEfpThreads) k_efp_distance(int n, const unsigned char* is_int, const double* a,
                                                              const double* b, double* part) {
    __shared__ double sh[kEfpThreads];
    double s = 0.0;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x)
        if (is_int[j]) s = __dadd_rn(s, fabs(__dsub_rn(a[j], b[j])));
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = kEfpThreads / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] = __dadd_rn(sh[threadIdx.x], sh[threadIdx.x + o]);
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__global__ void k_efp_distance_finish(const double* part, int nb, double* out) {
    if (threadIdx.x != 0) return;
    double s = 0.0;
    for (int b = 0; b < nb; ++b) s = __dadd_rn(s, part[b]);
    *out = s;
}

__global__ void k_efp_fill(int n, double v, double* a) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) a[i] = v;
}

__global__ void k_efp_cost_flag(int n, const double* __restrict__ c, int* __restrict__ flag) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) flag[j] = c[j] != 0.0;
}

// the cut row's entries: the nonzero costs in column order, after the problem's nnz entries
__global__ void k_efp_cut_entries(int n, const double* __restrict__ c, const int* __restrict__ pos, int nnz,
                                  int* __restrict__ col, double* __restrict__ val) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        const double cj = c[j];
        if (cj != 0.0) {
            col[nnz + pos[j]] = j;
            val[nnz + pos[j]] = cj;
        }
    }
}

__global__ void k_efp_cut_rows(int m, const int* __restrict__ rp, const double2* __restrict__ grow,
                               const int* __restrict__ ncost, int64_t* __restrict__ rp64, double* __restrict__ g) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k <= m + 1; k += gridDim.x * blockDim.x) {
        if (k <= m) rp64[k] = rp[k];
        else rp64[k] = (int64_t)rp[m] + *ncost;
        if (k < m) g[k] = grow[k].x;
    }
}

// out[0] = c x - delta, out[1] = c x: the sum in index order by one thread; delta = 1 when every
// nonzero cost sits on an integer variable and is integral, else 1e-4
__global__ void __launch_bounds__(kEfpThreads) k_efp_cut_rhs(int n, const double* __restrict__ c,
                                                             const unsigned char* __restrict__ is_int,
                                                             const double* __restrict__ x, double* out) {
    int any = 0, frac = 0;
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        const double cj = c[j];
        if (cj == 0.0) continue;
        any = 1;
        if (!is_int[j] || cj != floor(cj)) frac = 1;
    }
    any = __syncthreads_or(any);
    frac = __syncthreads_or(frac);
    if (threadIdx.x == 0) {
        double f = 0.0;
        for (int j = 0; j < n; ++j) f = __dadd_rn(f, __dmul_rn(c[j], x[j]));
        out[0] = __dsub_rn(f, any && !frac ? 1.0 : 1e-4);
        out[1] = f;
    }
}

}  // namespace gpubp

using namespace gpubp;

extern "C" void efp_params_default(efp_params* p) {
    if (!p) return;
    p->rounds = 20;
    p->lp_iterations = 500;
    p->ls_iterations = 200;
    p->cycle_window = 3;
    p->cycle_ratio = 0.1;
    p->seed = 1;
    p->improve = 0;
    p->polish = 0;
}

extern "C" int extended_fp(mip_problem* p, const double* lb, const double* ub, double* x_out, const efp_params* params,
                           efp_result* result, void* stream) {
    if (!p || !result || (p->n && (!lb || !ub || !x_out))) {
        set_error("extended_fp: null argument");
        return BP_ERR_INVALID;
    }
    efp_params prm;
    if (params) prm = *params;
    else efp_params_default(&prm);
    if (prm.rounds < 0 || prm.lp_iterations < 0 || prm.ls_iterations < 0 || prm.cycle_window < 1 ||
        !(prm.cycle_ratio >= 0.0) || (prm.improve != 0 && prm.improve != 1) || (prm.polish != 0 && prm.polish != 1)) {
        set_error("extended_fp: invalid parameters");
        return BP_ERR_INVALID;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const int n = p->n, m = p->m;
    const bool improve = prm.improve == 1;
    memset(result, 0, sizeof(*result));
    result->found_at = -3;
    result->status = 1;
    result->best_objective = INFINITY;
    std::vector<void*> tmp;
    mip_problem* q = p;   // the problem the loop works on: p, or p with the objective cut
    auto alloc_bytes = [&](void** ptr, size_t bytes) -> int {
        void* r = nullptr;
        cudaError_t e = cudaMallocAsync(&r, bytes ? bytes : 8, s);
        if (e != cudaSuccess) return fail_cuda(e, "cudaMallocAsync");
        tmp.push_back(r);
        *ptr = r;
        return BP_OK;
    };
    auto alloc = [&](double** ptr, size_t count) -> int {
        return alloc_bytes(reinterpret_cast<void**>(ptr), count * sizeof(double));
    };
    auto release = [&]() {
        if (q != p) {
            mip_free(q);
            q = p;
        }
        for (void* r : tmp) cudaFreeAsync(r, s);
        tmp.clear();
    };
#define EF_TRY(expr)           \
    do {                       \
        int _r = (expr);       \
        if (_r != BP_OK) {     \
            release();         \
            return _r;         \
        }                      \
    } while (0)
    // y, the weights and the ones carry one more entry for the cut row of the improvement mode
    double *x, *y, *xp, *sc, *s1, *s2, *w1, *w2, *c, *part, *dout, *ones_m, *xbest, *rhs, *xls = nullptr,
           *bls = nullptr;
    EF_TRY(alloc(&x, n));
    EF_TRY(alloc(&y, m + 1));
    EF_TRY(alloc(&xp, n));
    EF_TRY(alloc(&sc, n));
    EF_TRY(alloc(&s1, n));
    EF_TRY(alloc(&s2, n));
    EF_TRY(alloc(&w1, m + 1));
    EF_TRY(alloc(&w2, m + 1));
    EF_TRY(alloc(&c, n));
    EF_TRY(alloc(&part, kEfpBlocks));
    EF_TRY(alloc(&dout, 1));
    EF_TRY(alloc(&ones_m, m + 1));
    EF_TRY(alloc(&xbest, n));
    EF_TRY(alloc(&rhs, 2));
    if (improve && prm.polish) {
        EF_TRY(alloc(&xls, n));
        EF_TRY(alloc(&bls, n));
    }
    const int g = kEfpBlocks;
    auto fill = [&](double* a, int cnt, double v) { k_efp_fill<<<g, kEfpThreads, 0, s>>>(cnt, v, a); };
    auto copy = [&](double* dst, const double* src, int cnt) -> int {
        if (!cnt) return BP_OK;
        cudaError_t e = cudaMemcpyAsync(dst, src, sizeof(double) * (size_t)cnt, cudaMemcpyDeviceToDevice, s);
        return e == cudaSuccess ? BP_OK : fail_cuda(e, "cudaMemcpyAsync");
    };
    auto finish = [&](const double* point, int found_at) -> int {
        EF_TRY(copy(x_out, point, n));
        result->status = found_at >= -2 ? 0 : 1;
        result->found_at = found_at;
        return BP_OK;
    };
    // the cut problem's arrays, assembled at the first incumbent; the right-hand side changes
    int64_t* cut_rp = nullptr;
    int* cut_col = nullptr;
    double *cut_val = nullptr, *cut_g = nullptr;
    int ncost = 0;
    auto assemble_cut = [&]() -> int {
        int *flag, *pos, *dn;
        int rc;
        if ((rc = alloc_bytes(reinterpret_cast<void**>(&flag), sizeof(int) * (size_t)n)) != BP_OK ||
            (rc = alloc_bytes(reinterpret_cast<void**>(&pos), sizeof(int) * (size_t)n)) != BP_OK ||
            (rc = alloc_bytes(reinterpret_cast<void**>(&dn), sizeof(int))) != BP_OK ||
            (rc = alloc_bytes(reinterpret_cast<void**>(&cut_rp), sizeof(int64_t) * (size_t)(m + 2))) != BP_OK ||
            (rc = alloc_bytes(reinterpret_cast<void**>(&cut_col), sizeof(int) * (size_t)(p->nnz + n))) != BP_OK ||
            (rc = alloc(&cut_val, (size_t)(p->nnz + n))) != BP_OK || (rc = alloc(&cut_g, (size_t)(m + 1))) != BP_OK)
            return rc;
        k_efp_cost_flag<<<g, kEfpThreads, 0, s>>>(n, p->obj, flag);
        if ((rc = scan_exclusive(flag, pos, n, dn, s)) != BP_OK) return rc;
        k_efp_cut_entries<<<g, kEfpThreads, 0, s>>>(n, p->obj, pos, (int)p->nnz, cut_col, cut_val);
        k_efp_cut_rows<<<g, kEfpThreads, 0, s>>>(m, p->dp.row_ptr, p->dp.grow, dn, cut_rp, cut_g);
        cudaError_t e;
        if (p->nnz && ((e = cudaMemcpyAsync(cut_col, p->dp.col, sizeof(int) * (size_t)p->nnz, cudaMemcpyDeviceToDevice,
                                            s)) != cudaSuccess ||
                       (e = cudaMemcpyAsync(cut_val, p->dp.val, sizeof(double) * (size_t)p->nnz,
                                            cudaMemcpyDeviceToDevice, s)) != cudaSuccess))
            return fail_cuda(e, "cudaMemcpyAsync");
        if ((e = cudaMemcpyAsync(&ncost, dn, sizeof(int), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
            (e = cudaStreamSynchronize(s)) != cudaSuccess)
            return fail_cuda(e, "extended_fp cut row");
        return BP_OK;
    };
    // a new incumbent: the pump's first feasible point, or one of the cut problem
    double* W = nullptr;
    auto incumbent = [&](const double* pt, int where) -> int {
        int rc;
        if (result->improvements == 0) {
            result->status = 0;
            result->found_at = where;
            if ((rc = assemble_cut()) != BP_OK) return rc;
            if (cudaMemsetAsync(y + m, 0, sizeof(double), s) != cudaSuccess)
                return fail_cuda(cudaGetLastError(), "cudaMemsetAsync");
            fill(W + m, 1, 1.0);
        }
        if ((rc = copy(xbest, pt, n)) != BP_OK) return rc;
        if (prm.polish) {
            // the local search with its objective moves from the incumbent, on the problem
            // without the cut: its best when it recorded a later incumbent than its start
            ls_obj_params op{prm.ls_iterations, 0, 1.0};
            ls_obj_result orr;
            if ((rc = copy(xls, pt, n)) != BP_OK) return rc;
            fill(ones_m, m, 1.0);
            if ((rc = local_search_objective(p, lb, ub, xls, ones_m, bls, &op, &orr, stream)) != BP_OK) return rc;
            if (orr.improvements > 1) {
                if ((rc = copy(xbest, bls, n)) != BP_OK) return rc;
                result->polished += 1;
            }
        }
        result->improvements += 1;
        k_efp_cut_rhs<<<1, kEfpThreads, 0, s>>>(n, p->obj, p->dp.is_int, xbest, rhs);
        if ((rc = copy(cut_g + m, rhs, 1)) != BP_OK) return rc;
        double hr[2];
        cudaError_t e;
        if ((e = cudaMemcpyAsync(hr, rhs, sizeof(hr), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
            (e = cudaStreamSynchronize(s)) != cudaSuccess)
            return fail_cuda(e, "extended_fp cut");
        result->best_objective = hr[1];
        if (q != p) mip_free(q);
        q = p;
        mip_problem* nq = nullptr;
        rc = mip_load_csr(m + 1, n, cut_rp, cut_col, cut_val, cut_g, lb, ub, p->dp.is_int, p->obj, BP_MEM_DEVICE,
                          stream, &nq);
        if (rc != BP_OK) return rc;
        q = nq;
        return BP_OK;
    };
    pdhg_params pp;
    pdhg_params_default(&pp);
    pp.iterations = prm.lp_iterations;
    pp.restart_period = 100;
    pdhg_result pr;
    fp_params fpp;
    fp_params_default(&fpp);
    fp_result fr;
    ls_params lp{prm.ls_iterations, 0};
    ls_params lp_short{prm.ls_iterations / 5 > 0 ? prm.ls_iterations / 5 : 1, 0};
    ls_result r1, r2, rt;
    // start: the LP relaxation, rounded, then the local search
    k_efp_clip_zero<<<g, kEfpThreads, 0, s>>>(n, lb, ub, x);
    if (m && cudaMemsetAsync(y, 0, sizeof(double) * (size_t)m, s) != cudaSuccess) {
        release();
        return fail_cuda(cudaGetLastError(), "cudaMemsetAsync");
    }
    EF_TRY(pdhg_solve(p, lb, ub, x, y, &pp, &pr, stream));
    k_efp_snap<<<g, kEfpThreads, 0, s>>>(n, x, lb, ub, xp);
    fpp.seed = prm.seed;
    EF_TRY(fix_and_propagate(p, xp, lb, ub, nullptr, &fpp, s1, &fr, stream));
    fill(w1, m, 1.0);
    EF_TRY(local_search_mtm(p, lb, ub, s1, w1, &lp, &r1, stream));
    double* cur = s1;
    W = w1;
    bool start_found = false;
    if (r1.violated == 0) {
        if (!improve) {
            EF_TRY(finish(s1, -2));
            release();
            cudaStreamSynchronize(s);
            return BP_OK;
        }
        EF_TRY(incumbent(s1, -2));
        EF_TRY(copy(cur, xbest, n));   // the loop continues from the incumbent
        start_found = true;
    }
    if (!start_found) {
        k_efp_clip_zero<<<g, kEfpThreads, 0, s>>>(n, lb, ub, s2);
        fill(w2, m, 1.0);
        EF_TRY(local_search_mtm(p, lb, ub, s2, w2, &lp, &r2, stream));
        if (r2.violated == 0) {
            if (!improve) {
                EF_TRY(finish(s2, -1));
                release();
                cudaStreamSynchronize(s);
                return BP_OK;
            }
            cur = s2;
            W = w2;
            EF_TRY(incumbent(s2, -1));
            EF_TRY(copy(cur, xbest, n));
        } else if (r2.violated < r1.violated) {
            // the main loop's point and its kept weights: the start with fewer violated rows
            cur = s2;
            W = w2;
        }
    }
    std::vector<double> hist;
    for (int r = 0; r < prm.rounds; ++r) {
        const int mq = q->m;
        k_efp_objective<<<g, kEfpThreads, 0, s>>>(n, p->dp.is_int, cur, lb, ub, c);
        pp.objective = c;
        EF_TRY(pdhg_solve(q, lb, ub, x, y, &pp, &pr, stream));
        k_efp_snap<<<g, kEfpThreads, 0, s>>>(n, x, lb, ub, xp);
        k_efp_distance<<<g, kEfpThreads, 0, s>>>(n, p->dp.is_int, xp, cur, part);
        k_efp_distance_finish<<<1, 32, 0, s>>>(part, g, dout);
        double d = 0.0;
        if (cudaMemcpyAsync(&d, dout, sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess) {
            release();
            return fail_cuda(cudaGetLastError(), "extended_fp distance");
        }
        bool cyc = false;
        if ((int)hist.size() >= prm.cycle_window) {
            double sum = 0.0;
            for (size_t i = hist.size() - prm.cycle_window; i < hist.size(); ++i) sum += hist[i];
            const double mean = sum / prm.cycle_window;
            cyc = mean - d <= prm.cycle_ratio * mean;
        }
        hist.push_back(d);
        result->rounds = r + 1;
        result->last_distance = d;
        fpp.seed = prm.seed + (uint64_t)r + 1;
        EF_TRY(fix_and_propagate(q, xp, lb, ub, nullptr, &fpp, sc, &fr, stream));
        fill(ones_m, mq, 1.0);
        EF_TRY(local_search_mtm(q, lb, ub, sc, ones_m, &lp_short, &rt, stream));
        if (rt.violated == 0) {
            if (!improve) {
                EF_TRY(finish(sc, r));
                release();
                cudaStreamSynchronize(s);
                return BP_OK;
            }
            EF_TRY(incumbent(sc, r));
            EF_TRY(copy(cur, xbest, n));
            hist.clear();
            continue;
        }
        if (cyc) {
            EF_TRY(local_search_mtm(q, lb, ub, cur, W, &lp, &r1, stream));
            result->cycles++;
        } else {
            k_efp_nearest<<<g, kEfpThreads, 0, s>>>(n, p->dp.is_int, xp, lb, ub, cur);
        }
    }
    if (result->improvements > 0) {
        EF_TRY(copy(x_out, xbest, n));
    } else {
        EF_TRY(copy(x_out, cur, n));
    }
    release();
    if (cudaStreamSynchronize(s) != cudaSuccess) return fail_cuda(cudaGetLastError(), "extended_fp");
    p->last_stream = s;
    return BP_OK;
#undef EF_TRY
}
