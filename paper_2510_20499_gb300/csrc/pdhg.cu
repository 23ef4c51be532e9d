// The approximate LP (Sections 1 and 2.5: the paper's GPU PDLP): warm-started primal-dual
// hybrid gradient for
//     min c^T x   subject to   A x <= g,   l <= x <= u        (rows with g = +inf are free)
// with row duals y >= 0:
//     x+ = proj_[l, u](x - tau (c + A^T y)),      xe = 2 x+ - x,
//     y+ = max(0, y + sigma (A xe - g)),          tau = eta / omega, sigma = eta * omega,
// and, with a restart period R > 0, every R iterations the iterate replaced by the mean of the
// period's R iterates (a fixed period: every step is a plain function of the inputs).  Default
// eta = 0.9 / sqrt(max column |a| sum * max row |a| sum) (a bound on ||A||_2), default primal
// weight omega = ||c||_2 / ||g||_2 over the finite rows (PDLP's initial weight).
//
// One iteration streams the matrix twice (one fused multiply-add per nonzero: this part's FP64
// rate, about 1.7 lane-operations per SM and clock, is the other bound besides HBM):
//   k_pdhg_cols   a thread per column over the transpose (row_idx, col_val): A^T y, fused
//                 with the x step, the extrapolation and the restart sums;
//   k_pdhg_rows   a flat task space over the row classes of the handle: a warp per piece of a
//                 long row (partial sum into its slot), a warp per warp row, a thread per
//                 thread row; finished rows take the y step at once;
//   k_pdhg_long   a warp per long row sums its pieces' partials in slot order, then the y step.
// The same kernels with `eval` set produce A x and c + A^T y for the KKT measures; every sum over
// a row, a column or the whole problem has a fixed order, so repeated runs are bit-identical.
#include <climits>
#include <cmath>

#include "bp_host.h"

namespace gpubp {

constexpr int kPdThreads = 256;
constexpr int kPdRedBlocks = 304;         // blocks of the reductions (fixed: a fixed order)

struct PdhgVecs {
    const double* c;
    const double* l;
    const double* u;
    double tau, sigma;
};

// ---------------------------------------------------------------- column pass
// x+ = clamp(x - tau (c + A^T y), l, u), xe = 2 x+ - x, xs += x+ (restart sums, when given).
// eval: r = c + A^T y into xn (nothing else).
__global__ void __launch_bounds__(kPdThreads) k_pdhg_cols(DevProblem P, PdhgVecs V, const double* __restrict__ x,
                                                          const double* __restrict__ y, double* __restrict__ xn,
                                                          double* __restrict__ xe, double* __restrict__ xs, int eval) {
    // a thread per column: 32 columns in flight per warp, the column's own vectors loaded
    // before its sum, the sum's loads unrolled (independent of each other)
    const int stride = gridDim.x * blockDim.x;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < P.n; j += stride) {
        const int b = P.col_ptr[j], e = P.col_ptr[j + 1];
        const double cj = V.c[j];
        double xj = 0.0, lj = 0.0, uj = 0.0, sj = 0.0;
        if (!eval) {
            xj = x[j];
            lj = V.l[j];
            uj = V.u[j];
            if (xs) sj = xs[j];
        }
        double s = 0.0;
        int q = b;
        for (; q + 4 <= e; q += 4) {
            const int r0 = P.row_idx[q], r1 = P.row_idx[q + 1], r2 = P.row_idx[q + 2], r3 = P.row_idx[q + 3];
            const double a0 = P.col_val[q], a1 = P.col_val[q + 1], a2 = P.col_val[q + 2], a3 = P.col_val[q + 3];
            const double y0 = y[r0], y1 = y[r1], y2 = y[r2], y3 = y[r3];
            s = fma(a0, y0, s);
            s = fma(a1, y1, s);
            s = fma(a2, y2, s);
            s = fma(a3, y3, s);
        }
        for (; q < e; ++q) s = fma(P.col_val[q], y[P.row_idx[q]], s);
        const double r = __dadd_rn(cj, s);
        if (eval) {
            xn[j] = r;
        } else {
            double v = __dsub_rn(xj, __dmul_rn(V.tau, r));
            v = v < lj ? lj : v;   // max(v, l), then min(., u)
            v = v > uj ? uj : v;
            xn[j] = v;
            xe[j] = __dsub_rn(__dmul_rn(2.0, v), xj);
            if (xs) xs[j] = __dadd_rn(sj, v);
        }
    }
}

// the y step of row k from its sum s = (A xe)_k; eval: A x into yn
__device__ __forceinline__ void pdhg_row_done(const DevProblem& P, const PdhgVecs& V, int k, double s, const double* y,
                                              double* yn, double* ys, int eval) {
    if (eval) {
        yn[k] = s;
        return;
    }
    const double v = __dadd_rn(y[k], __dmul_rn(V.sigma, __dsub_rn(s, P.grow[k].x)));
    const double w = v > 0.0 ? v : 0.0;
    yn[k] = w;
    if (ys) ys[k] = __dadd_rn(ys[k], w);
}

// ---------------------------------------------------------------- row pass
// This lane's share of sum over [beg, end) of val * v[col] (nonzeros lane, lane + 32, ...).
__device__ __forceinline__ double warp_dot(const DevProblem& P, const double* __restrict__ v, int beg, int end,
                                           int lane) {
    double s = 0.0;
    for (int q = beg + lane; q < end; q += 32) s = fma(P.val[q], v[P.col[q]], s);
    return s;
}

// Warp tasks [pieces of long rows][warp rows][thread rows in groups of 32]: pieces write their
// partial sums (slot = the piece's index in the round-0 piece list), the others finish their
// rows.
__global__ void __launch_bounds__(kPdThreads) k_pdhg_rows(DevProblem P, PdhgVecs V, const double* __restrict__ xe,
                                                          const double* __restrict__ y, double* __restrict__ yn,
                                                          double* __restrict__ ys, double* __restrict__ part, int eval) {
    const int lane = threadIdx.x & 31;
    const int nwarp_rows = P.class_off[kClassWarpRow + 1] - P.class_off[kClassWarpRow];
    const int nthread_rows = P.class_off[kNumThreadBins] - P.class_off[0];
    const int t_pieces = P.npieces, t_warp = nwarp_rows, t_thread = (nthread_rows + 31) / 32;
    const int total = t_pieces + t_warp + t_thread;
    const int NW = (gridDim.x * blockDim.x) >> 5;
    for (int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; t < total; t += NW) {
        if (t < t_pieces) {
            const int4 tk = P.static_tasks[t];
            const int beg = tk.z, end = min(tk.w, tk.z + P.chunk_len);
            const double s0 = warp_dot(P, xe, beg, end, lane);
            double s = s0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s = __dadd_rn(s, __shfl_xor_sync(0xffffffffu, s, o));
            if (lane == 0) part[t] = s;
        } else if (t < t_pieces + t_warp) {
            const int k = P.static_list[P.class_off[kClassWarpRow] + (t - t_pieces)];
            double s = warp_dot(P, xe, P.row_ptr[k], P.row_ptr[k + 1], lane);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s = __dadd_rn(s, __shfl_xor_sync(0xffffffffu, s, o));
            if (lane == 0) pdhg_row_done(P, V, k, s, y, yn, ys, eval);
        } else {
            const int i = (t - t_pieces - t_warp) * 32 + lane;
            if (i < nthread_rows) {
                const int k = P.static_list[P.class_off[0] + i];
                const int e = P.row_ptr[k + 1];
                double s = 0.0;
                int q = P.row_ptr[k];
                // four nonzeros' loads issued together; the sum keeps the row order
                for (; q + 4 <= e; q += 4) {
                    const int c0 = P.col[q], c1 = P.col[q + 1], c2 = P.col[q + 2], c3 = P.col[q + 3];
                    const double a0 = P.val[q], a1 = P.val[q + 1], a2 = P.val[q + 2], a3 = P.val[q + 3];
                    const double v0 = xe[c0], v1 = xe[c1], v2 = xe[c2], v3 = xe[c3];
                    s = fma(a0, v0, s);
                    s = fma(a1, v1, s);
                    s = fma(a2, v2, s);
                    s = fma(a3, v3, s);
                }
                for (; q < e; ++q) s = fma(P.val[q], xe[P.col[q]], s);
                pdhg_row_done(P, V, k, s, y, yn, ys, eval);
            }
        }
    }
}

// A warp per long row (its first piece's descriptor): the partials of its pieces in slot order
// (lanes strided, then a fixed reduction), then the y step.
__global__ void __launch_bounds__(kPdThreads) k_pdhg_long(DevProblem P, PdhgVecs V, const double* __restrict__ part,
                                                          const double* __restrict__ y, double* __restrict__ yn,
                                                          double* __restrict__ ys, int eval) {
    const int lane = threadIdx.x & 31;
    const int NW = (gridDim.x * blockDim.x) >> 5;
    for (int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; t < P.npieces; t += NW) {
        const int4 tk = P.static_tasks[t];
        if (tk.y != 0) continue;   // not the row's first piece
        const int npc = (tk.w - tk.z + P.chunk_len - 1) / P.chunk_len;
        double s = 0.0;
        for (int i = lane; i < npc; i += 32) s = __dadd_rn(s, part[t + i]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s = __dadd_rn(s, __shfl_xor_sync(0xffffffffu, s, o));
        if (lane == 0) pdhg_row_done(P, V, tk.x, s, y, yn, ys, eval);
    }
}

// ---------------------------------------------------------------- Ruiz preconditioning
// A pass computes the largest scaled |a| = (D_r |a|) D_c of every row (a warp per row) and of
// every column (a thread per column over the transpose) from the same factors, then divides
// each factor by the square root of its maximum (factor kept where the maximum is 0).
__global__ void __launch_bounds__(kPdThreads) k_ruiz_rows(DevProblem P, const double* __restrict__ Dr,
                                                          const double* __restrict__ Dc, double* __restrict__ R) {
    const int lane = threadIdx.x & 31;
    for (int k = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; k < P.m; k += (gridDim.x * blockDim.x) >> 5) {
        double mx = 0.0;
        for (int q = P.row_ptr[k] + lane; q < P.row_ptr[k + 1]; q += 32)
            mx = fmax(mx, __dmul_rn(__dmul_rn(Dr[k], fabs(P.val[q])), Dc[P.col[q]]));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if (lane == 0) R[k] = mx;
    }
}

__global__ void __launch_bounds__(kPdThreads) k_ruiz_cols(DevProblem P, const double* __restrict__ Dr,
                                                          const double* __restrict__ Dc, double* __restrict__ C) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < P.n; j += gridDim.x * blockDim.x) {
        double mx = 0.0;
        for (int c = P.col_ptr[j]; c < P.col_ptr[j + 1]; ++c)
            mx = fmax(mx, __dmul_rn(__dmul_rn(Dr[P.row_idx[c]], fabs(P.col_val[c])), Dc[j]));
        C[j] = mx;
    }
}

__global__ void k_ruiz_update(int cnt, double* __restrict__ D, const double* __restrict__ M) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += gridDim.x * blockDim.x)
        if (M[i] > 0.0) D[i] = __ddiv_rn(D[i], sqrt(M[i]));
}

// the scaled matrix (D_r a) D_c in both layouts, the scaled right-hand sides D_r g
__global__ void __launch_bounds__(kPdThreads) k_scale_rows(DevProblem P, const double* __restrict__ Dr,
                                                           const double* __restrict__ Dc, double* __restrict__ sval,
                                                           double2* __restrict__ sgrow) {
    const int lane = threadIdx.x & 31;
    for (int k = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; k < P.m; k += (gridDim.x * blockDim.x) >> 5) {
        for (int q = P.row_ptr[k] + lane; q < P.row_ptr[k + 1]; q += 32)
            sval[q] = __dmul_rn(__dmul_rn(Dr[k], P.val[q]), Dc[P.col[q]]);
        if (lane == 0) {
            const double g = __dmul_rn(Dr[k], P.grow[k].x);
            sgrow[k] = make_double2(g, g);
        }
    }
}

__global__ void __launch_bounds__(kPdThreads) k_scale_cols(DevProblem P, const double* __restrict__ Dr,
                                                           const double* __restrict__ Dc, double* __restrict__ scol) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < P.n; j += gridDim.x * blockDim.x)
        for (int c = P.col_ptr[j]; c < P.col_ptr[j + 1]; ++c)
            scol[c] = __dmul_rn(__dmul_rn(Dr[P.row_idx[c]], P.col_val[c]), Dc[j]);
}

// D_c c, l / D_c, u / D_c and the warm start x / D_c
__global__ void k_scale_cvecs(int n, const double* __restrict__ Dc, const double* __restrict__ c,
                              const double* __restrict__ l, const double* __restrict__ u, double* __restrict__ cs,
                              double* __restrict__ ls, double* __restrict__ us, double* __restrict__ x) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        const double d = Dc[j];
        cs[j] = __dmul_rn(d, c[j]);
        ls[j] = __ddiv_rn(l[j], d);
        us[j] = __ddiv_rn(u[j], d);
        x[j] = __ddiv_rn(x[j], d);
    }
}

// v = v / D (into the scaled space) or v = D v (back)
__global__ void k_scale_vec(int cnt, const double* __restrict__ D, double* __restrict__ v, int back) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += gridDim.x * blockDim.x)
        v[i] = back ? __dmul_rn(D[i], v[i]) : __ddiv_rn(v[i], D[i]);
}

__global__ void k_pdhg_fill(int cnt, double v, double* __restrict__ a) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += gridDim.x * blockDim.x) a[i] = v;
}

// restart: (x, y) = (xs, ys) / R, sums cleared
__global__ void k_pdhg_restart(int n, int m, double r, double* x, double* y, double* xs, double* ys) {
    const int stride = gridDim.x * blockDim.x;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += stride) {
        x[j] = __ddiv_rn(xs[j], r);
        xs[j] = 0.0;
    }
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < m; k += stride) {
        y[k] = __ddiv_rn(ys[k], r);
        ys[k] = 0.0;
    }
}

// ---------------------------------------------------------------- reductions (fixed order)
// Block sums of up to 5 values per thread into part[5 * block + i]: a fixed tree per block.
__device__ void block_sum5(double v[5], double* part) {
    __shared__ double sh[5][kPdThreads];
    for (int i = 0; i < 5; ++i) sh[i][threadIdx.x] = v[i];
    __syncthreads();
    for (int o = kPdThreads / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o)
            for (int i = 0; i < 5; ++i) sh[i][threadIdx.x] = __dadd_rn(sh[i][threadIdx.x], sh[i][threadIdx.x + o]);
        __syncthreads();
    }
    if (threadIdx.x < 5) part[5 * blockIdx.x + threadIdx.x] = sh[threadIdx.x][0];
}

// Step-size inputs: [0] max column |a| sum, [1] max row |a| sum (per block maxima), [2] sum of c^2,
// [3] sum of g^2 over finite rows (per block sums).  A thread per column, a warp per row.
__global__ void __launch_bounds__(kPdThreads) k_pdhg_norms(DevProblem P, const double* c, double* part) {
    const int tid = blockIdx.x * blockDim.x + threadIdx.x, stride = gridDim.x * blockDim.x;
    const int lane = threadIdx.x & 31;
    double v[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    for (int j = tid; j < P.n; j += stride) {
        double s = 0.0;
        for (int q = P.col_ptr[j]; q < P.col_ptr[j + 1]; ++q) s = __dadd_rn(s, fabs(P.col_val[q]));
        v[0] = s > v[0] ? s : v[0];
        v[2] = __dadd_rn(v[2], __dmul_rn(c[j], c[j]));
    }
    for (int k = tid >> 5; k < P.m; k += stride >> 5) {
        double s = 0.0;
        for (int q = P.row_ptr[k] + lane; q < P.row_ptr[k + 1]; q += 32) s = __dadd_rn(s, fabs(P.val[q]));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s = __dadd_rn(s, __shfl_xor_sync(0xffffffffu, s, o));
        if (lane == 0) {
            v[1] = s > v[1] ? s : v[1];
            const double g = P.grow[k].x;
            if (isfinite(g)) v[3] = __dadd_rn(v[3], __dmul_rn(g, g));
        }
    }
    // maxima through the sum tree would be wrong: reduce them separately
    __shared__ double mx[2][kPdThreads];
    mx[0][threadIdx.x] = v[0];
    mx[1][threadIdx.x] = v[1];
    __syncthreads();
    for (int o = kPdThreads / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o)
            for (int i = 0; i < 2; ++i) mx[i][threadIdx.x] = fmax(mx[i][threadIdx.x], mx[i][threadIdx.x + o]);
        __syncthreads();
    }
    // the block maxima enter the same tree from thread 0 (adding zeros is exact)
    v[0] = threadIdx.x == 0 ? mx[0][0] : 0.0;
    v[1] = threadIdx.x == 0 ? mx[1][0] : 0.0;
    block_sum5(v, part);
}

// KKT sums: [0] sum over finite rows of max(Ax - g, 0)^2, [1] sum over finite rows of g y,
// [2] c^T x, [3] sum of the squared reduced costs pushing toward an infinite bound, [4] sum of
// the finite parts of min over [l, u] of r_j x_j (Ax in ax, r = c + A^T y in r).
__global__ void __launch_bounds__(kPdThreads) k_pdhg_kkt(DevProblem P, const double* c, const double* l,
                                                         const double* u, const double* x, const double* y,
                                                         const double* ax, const double* r, double* part) {
    const int tid = blockIdx.x * blockDim.x + threadIdx.x, stride = gridDim.x * blockDim.x;
    double v[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    for (int k = tid; k < P.m; k += stride) {
        const double g = P.grow[k].x;
        if (!isfinite(g)) continue;
        const double d = __dsub_rn(ax[k], g);
        if (d > 0.0) v[0] = __dadd_rn(v[0], __dmul_rn(d, d));
        v[1] = __dadd_rn(v[1], __dmul_rn(g, y[k]));
    }
    for (int j = tid; j < P.n; j += stride) {
        v[2] = __dadd_rn(v[2], __dmul_rn(c[j], x[j]));
        const double rj = r[j];
        const bool lf = isfinite(l[j]), uf = isfinite(u[j]);
        if (rj > 0.0 && !lf) v[3] = __dadd_rn(v[3], __dmul_rn(rj, rj));
        if (rj < 0.0 && !uf) v[3] = __dadd_rn(v[3], __dmul_rn(rj, rj));
        v[4] = __dadd_rn(v[4], rj > 0.0 ? __dmul_rn(rj, lf ? l[j] : 0.0) : __dmul_rn(rj, uf ? u[j] : 0.0));
    }
    block_sum5(v, part);
}

// sums (or, for the step inputs' first two, maxima) of the blocks' partials: thread t takes
// blocks t, t + 256, ..., then a fixed tree (one block of kPdThreads threads)
__global__ void __launch_bounds__(kPdThreads) k_pdhg_finish(const double* part, int nblocks, int maxima, double* out) {
    __shared__ double sh[5][kPdThreads];
    for (int i = 0; i < 5; ++i) {
        const bool mx = maxima && i < 2;
        double s = 0.0;
        for (int b = threadIdx.x; b < nblocks; b += kPdThreads) {
            const double v = part[5 * b + i];
            s = mx ? fmax(s, v) : __dadd_rn(s, v);
        }
        sh[i][threadIdx.x] = s;
    }
    __syncthreads();
    for (int o = kPdThreads / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o)
            for (int i = 0; i < 5; ++i) {
                const bool mx = maxima && i < 2;
                sh[i][threadIdx.x] = mx ? fmax(sh[i][threadIdx.x], sh[i][threadIdx.x + o])
                                        : __dadd_rn(sh[i][threadIdx.x], sh[i][threadIdx.x + o]);
            }
        __syncthreads();
    }
    if (threadIdx.x < 5) out[threadIdx.x] = sh[threadIdx.x][0];
}

}  // namespace gpubp

using namespace gpubp;

extern "C" void pdhg_params_default(pdhg_params* p) {
    if (!p) return;
    p->iterations = 1000;
    p->restart_period = 100;
    p->step = 0.0;
    p->primal_weight = 0.0;
    p->objective = nullptr;
    p->scaling_iterations = 0;
    p->reserved = 0;
}

extern "C" int pdhg_solve(mip_problem* p, const double* lb, const double* ub, double* x, double* y,
                          const pdhg_params* params, pdhg_result* result, void* stream) {
    if (!p || !result || (p->n && (!lb || !ub || !x)) || (p->m && !y)) {
        set_error("pdhg_solve: null argument");
        return BP_ERR_INVALID;
    }
    pdhg_params prm;
    if (params) prm = *params;
    else pdhg_params_default(&prm);
    if (prm.iterations < 0 || prm.restart_period < 0 || !(prm.step >= 0.0) || !(prm.primal_weight >= 0.0) ||
        prm.scaling_iterations < 0) {
        set_error("pdhg_solve: invalid parameters");
        return BP_ERR_INVALID;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const int n = p->n, m = p->m, np_ = p->dp.npieces;
    const double* cobj = prm.objective ? prm.objective : p->obj;
    memset(result, 0, sizeof(*result));
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
#define PD_TRY(expr)                       \
    do {                                   \
        int _r = (expr);                   \
        if (_r != BP_OK) {                 \
            release();                     \
            return _r;                     \
        }                                  \
    } while (0)
#define PD_CUDA(expr)                                      \
    do {                                                   \
        cudaError_t _e = (expr);                           \
        if (_e != cudaSuccess) {                           \
            release();                                     \
            return fail_cuda(_e, #expr);                   \
        }                                                  \
    } while (0)
    const bool restarts = prm.restart_period > 0;
    double *xn, *xe, *yn, *part, *xs = nullptr, *ys = nullptr, *red, *sums;
    PD_TRY(alloc(&xn, (size_t)n));
    PD_TRY(alloc(&xe, (size_t)n));
    PD_TRY(alloc(&yn, (size_t)m));
    PD_TRY(alloc(&part, (size_t)np_));
    PD_TRY(alloc(&red, 5 * (size_t)kPdRedBlocks));
    PD_TRY(alloc(&sums, 5));
    if (restarts) {
        PD_TRY(alloc(&xs, (size_t)n));
        PD_TRY(alloc(&ys, (size_t)m));
        PD_CUDA(cudaMemsetAsync(xs, 0, sizeof(double) * (size_t)n, s));
        PD_CUDA(cudaMemsetAsync(ys, 0, sizeof(double) * (size_t)m, s));
    }
    double hs[5];
    // Ruiz preconditioning: the iteration runs on the scaled problem (Ps, cv, lv, uv) from the
    // scaled warm start; the final measures use the original one
    DevProblem Ps = p->dp;
    const double *cv = cobj, *lv = lb, *uv = ub;
    double *Dr = nullptr, *Dc = nullptr;
    const int K = prm.scaling_iterations;
    if (K > 0) {
        double *R, *Cm, *sval, *scol, *sgrow, *cs, *ls, *us;
        PD_TRY(alloc(&Dr, (size_t)m));
        PD_TRY(alloc(&Dc, (size_t)n));
        PD_TRY(alloc(&R, (size_t)m));
        PD_TRY(alloc(&Cm, (size_t)n));
        PD_TRY(alloc(&sval, (size_t)p->nnz));
        PD_TRY(alloc(&scol, (size_t)p->nnz));
        PD_TRY(alloc(&sgrow, 2 * (size_t)m));
        PD_TRY(alloc(&cs, (size_t)n));
        PD_TRY(alloc(&ls, (size_t)n));
        PD_TRY(alloc(&us, (size_t)n));
        const int gr = p->sms * 8;
        k_pdhg_fill<<<gr, kPdThreads, 0, s>>>(m, 1.0, Dr);
        k_pdhg_fill<<<gr, kPdThreads, 0, s>>>(n, 1.0, Dc);
        for (int k = 0; k < K; ++k) {
            k_ruiz_rows<<<gr, kPdThreads, 0, s>>>(p->dp, Dr, Dc, R);
            k_ruiz_cols<<<gr, kPdThreads, 0, s>>>(p->dp, Dr, Dc, Cm);
            k_ruiz_update<<<gr, kPdThreads, 0, s>>>(m, Dr, R);
            k_ruiz_update<<<gr, kPdThreads, 0, s>>>(n, Dc, Cm);
        }
        k_scale_rows<<<gr, kPdThreads, 0, s>>>(p->dp, Dr, Dc, sval, reinterpret_cast<double2*>(sgrow));
        k_scale_cols<<<gr, kPdThreads, 0, s>>>(p->dp, Dr, Dc, scol);
        k_scale_cvecs<<<gr, kPdThreads, 0, s>>>(n, Dc, cobj, lb, ub, cs, ls, us, x);
        k_scale_vec<<<gr, kPdThreads, 0, s>>>(m, Dr, y, 0);
        PD_CUDA(cudaGetLastError());
        Ps.val = sval;
        Ps.col_val = scol;
        Ps.grow = reinterpret_cast<const double2*>(sgrow);
        cv = cs;
        lv = ls;
        uv = us;
    }
    // step and primal weight
    double eta = prm.step, omega = prm.primal_weight;
    if (eta == 0.0 || omega == 0.0) {
        k_pdhg_norms<<<kPdRedBlocks, kPdThreads, 0, s>>>(Ps, cv, red);
        k_pdhg_finish<<<1, kPdThreads, 0, s>>>(red, kPdRedBlocks, 1, sums);
        PD_CUDA(cudaGetLastError());
        PD_CUDA(cudaMemcpyAsync(hs, sums, sizeof(hs), cudaMemcpyDeviceToHost, s));
        PD_CUDA(cudaStreamSynchronize(s));
        if (eta == 0.0) eta = (hs[0] > 0.0 && hs[1] > 0.0) ? 0.9 / std::sqrt(hs[0] * hs[1]) : 1.0;
        if (omega == 0.0) {
            const double nc = std::sqrt(hs[2]), ng = std::sqrt(hs[3]);
            omega = (nc > 0.0 && ng > 0.0) ? nc / ng : 1.0;
        }
    }
    PdhgVecs V{cv, lv, uv, eta / omega, eta * omega};
    const PdhgVecs V0{cobj, lb, ub, eta / omega, eta * omega};   // the original problem's vectors
    // grids of resident blocks (every block stays resident through its grid-stride loop)
    static int occ[3] = {-1, -1, -1};
    if (occ[0] < 0) {
        PD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ[0], k_pdhg_cols, kPdThreads, 0));
        PD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ[1], k_pdhg_rows, kPdThreads, 0));
        PD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ[2], k_pdhg_long, kPdThreads, 0));
    }
    const int grid_c = p->sms * (occ[0] > 0 ? occ[0] : 1), grid = p->sms * (occ[1] > 0 ? occ[1] : 1);
    const int grid_l = p->sms * (occ[2] > 0 ? occ[2] : 1);
    double *xc = x, *xo = xn, *yc = y, *yo = yn;
    int restarts_done = 0;
    for (int it = 0; it < prm.iterations; ++it) {
        k_pdhg_cols<<<grid_c, kPdThreads, 0, s>>>(Ps, V, xc, yc, xo, xe, xs, 0);
        k_pdhg_rows<<<grid, kPdThreads, 0, s>>>(Ps, V, xe, yc, yo, ys, part, 0);
        if (np_) k_pdhg_long<<<grid_l, kPdThreads, 0, s>>>(Ps, V, part, yc, yo, ys, 0);
        std::swap(xc, xo);
        std::swap(yc, yo);
        if (restarts && (it + 1) % prm.restart_period == 0) {
            k_pdhg_restart<<<grid, kPdThreads, 0, s>>>(n, m, (double)prm.restart_period, xc, yc, xs, ys);
            ++restarts_done;
        }
    }
    PD_CUDA(cudaGetLastError());
    if (xc != x && n) PD_CUDA(cudaMemcpyAsync(x, xc, sizeof(double) * (size_t)n, cudaMemcpyDeviceToDevice, s));
    if (yc != y && m) PD_CUDA(cudaMemcpyAsync(y, yc, sizeof(double) * (size_t)m, cudaMemcpyDeviceToDevice, s));
    if (K > 0) {   // back to the original variables: x = D_c x~, y = D_r y~
        k_scale_vec<<<p->sms * 8, kPdThreads, 0, s>>>(n, Dc, x, 1);
        k_scale_vec<<<p->sms * 8, kPdThreads, 0, s>>>(m, Dr, y, 1);
    }
    // KKT measures of the final iterate (original problem): A x into yn, c + A^T y into xn
    k_pdhg_rows<<<grid, kPdThreads, 0, s>>>(p->dp, V0, x, y, yn, nullptr, part, 1);
    if (np_) k_pdhg_long<<<grid_l, kPdThreads, 0, s>>>(p->dp, V0, part, y, yn, nullptr, 1);
    k_pdhg_cols<<<grid_c, kPdThreads, 0, s>>>(p->dp, V0, x, y, xn, xe, nullptr, 1);
    k_pdhg_kkt<<<kPdRedBlocks, kPdThreads, 0, s>>>(p->dp, cobj, lb, ub, x, y, yn, xn, red);
    k_pdhg_finish<<<1, kPdThreads, 0, s>>>(red, kPdRedBlocks, 0, sums);
    PD_CUDA(cudaGetLastError());
    PD_CUDA(cudaMemcpyAsync(hs, sums, sizeof(hs), cudaMemcpyDeviceToHost, s));
    release();
    PD_CUDA(cudaStreamSynchronize(s));
    result->iterations = prm.iterations;
    result->restarts = restarts_done;
    result->step = eta;
    result->primal_weight = omega;
    result->primal_residual = std::sqrt(hs[0]);
    result->dual_residual = std::sqrt(hs[3]);
    result->primal_obj = hs[2];
    result->dual_obj = -hs[1] + hs[4];
    p->last_stream = s;
    return BP_OK;
#undef PD_TRY
#undef PD_CUDA
}
