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
        !(prm.cycle_ratio >= 0.0)) {
        set_error("extended_fp: invalid parameters");
        return BP_ERR_INVALID;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const int n = p->n, m = p->m;
    memset(result, 0, sizeof(*result));
    result->found_at = -3;
    result->status = 1;
    std::vector<void*> tmp;
    auto alloc = [&](double** ptr, size_t count) -> int {
        void* q = nullptr;
        cudaError_t e = cudaMallocAsync(&q, (count ? count : 1) * sizeof(double), s);
        if (e != cudaSuccess) return fail_cuda(e, "cudaMallocAsync");
        tmp.push_back(q);
        *ptr = static_cast<double*>(q);
        return BP_OK;
    };
    auto release = [&]() {
        for (void* q : tmp) cudaFreeAsync(q, s);
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
    double *x, *y, *xp, *sc, *s1, *s2, *w1, *w2, *c, *part, *dout, *ones_m;
    EF_TRY(alloc(&x, n));
    EF_TRY(alloc(&y, m));
    EF_TRY(alloc(&xp, n));
    EF_TRY(alloc(&sc, n));
    EF_TRY(alloc(&s1, n));
    EF_TRY(alloc(&s2, n));
    EF_TRY(alloc(&w1, m));
    EF_TRY(alloc(&w2, m));
    EF_TRY(alloc(&c, n));
    EF_TRY(alloc(&part, kEfpBlocks));
    EF_TRY(alloc(&dout, 1));
    EF_TRY(alloc(&ones_m, m));
    const int g = kEfpBlocks;
    auto fill_ones = [&](double* a) { k_efp_fill<<<g, kEfpThreads, 0, s>>>(m, 1.0, a); };
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
    fill_ones(w1);
    EF_TRY(local_search_mtm(p, lb, ub, s1, w1, &lp, &r1, stream));
    if (r1.violated == 0) {
        EF_TRY(finish(s1, -2));
        release();
        cudaStreamSynchronize(s);
        return BP_OK;
    }
    k_efp_clip_zero<<<g, kEfpThreads, 0, s>>>(n, lb, ub, s2);
    fill_ones(w2);
    EF_TRY(local_search_mtm(p, lb, ub, s2, w2, &lp, &r2, stream));
    if (r2.violated == 0) {
        EF_TRY(finish(s2, -1));
        release();
        cudaStreamSynchronize(s);
        return BP_OK;
    }
    // the main loop's point and its kept weights: the start with fewer violated rows
    double* cur = r2.violated < r1.violated ? s2 : s1;
    double* W = r2.violated < r1.violated ? w2 : w1;
    std::vector<double> hist;
    for (int r = 0; r < prm.rounds; ++r) {
        k_efp_objective<<<g, kEfpThreads, 0, s>>>(n, p->dp.is_int, cur, lb, ub, c);
        pp.objective = c;
        EF_TRY(pdhg_solve(p, lb, ub, x, y, &pp, &pr, stream));
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
        EF_TRY(fix_and_propagate(p, xp, lb, ub, nullptr, &fpp, sc, &fr, stream));
        fill_ones(ones_m);
        EF_TRY(local_search_mtm(p, lb, ub, sc, ones_m, &lp_short, &rt, stream));
        if (rt.violated == 0) {
            EF_TRY(finish(sc, r));
            release();
            cudaStreamSynchronize(s);
            return BP_OK;
        }
        if (cyc) {
            EF_TRY(local_search_mtm(p, lb, ub, cur, W, &lp, &r1, stream));
            result->cycles++;
        } else {
            k_efp_nearest<<<g, kEfpThreads, 0, s>>>(n, p->dp.is_int, xp, lb, ub, cur);
        }
    }
    EF_TRY(finish(cur, -3));
    release();
    if (cudaStreamSynchronize(s) != cudaSuccess) return fail_cuda(cudaGetLastError(), "extended_fp");
    p->last_stream = s;
    return BP_OK;
#undef EF_TRY
}
