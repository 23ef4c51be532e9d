// Probe priority (Section 2.2): bp_probe_priority.
//
// The paper ranks the variables to probe by three keys, lexicographically: the number of rows
// a variable would violate if its contribution to the minimal activity flipped from its
// minimising to its maximising bound (only variables whose coefficients have both signs),
// the largest such violation, and the smallest unit slack (g - L_min) / |a| over its rows.
// One warp per row computes the minimal activities, one warp per variable walks its column of
// the transpose, and three stable radix passes (key3 ascending, key2 descending, key1
// descending; the input is in index order) give the order.
#include <climits>

#include "bp_host.h"

namespace gpubp {

__global__ void k_row_minact(DevProblem P, const longlong2* bk, double* minfin, int* ninf) {
    const int lane = threadIdx.x & 31;
    for (int k = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; k < P.m; k += (gridDim.x * blockDim.x) >> 5) {
        double s = 0.0;
        int c = 0;
        for (int q = P.row_ptr[k] + lane; q < P.row_ptr[k + 1]; q += 32) {
            const double a = P.val[q];
            const longlong2 b = bk[P.col[q]];
            const long long key = a > 0 ? b.x : b.y;
            if (key_is_inf(key)) ++c;
            else s = fma(a, kdec(key), s);
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

// is the variable probed (integer, l < u, at least one finite bound)?
__device__ __forceinline__ bool probeable(bool is_i, long long lk, long long uk) {
    return is_i && lk < uk && !(lk == kKeyNegInf && uk == kKeyPosInf);
}

__global__ void k_var_keys(DevProblem P, const longlong2* bk, const double* minfin, const int* ninf, int* key1,
                           double* key2, double* key3, int* flag) {
    const int lane = threadIdx.x & 31;
    for (int v = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; v < P.n; v += (gridDim.x * blockDim.x) >> 5) {
        const longlong2 b = bk[v];
        if (!probeable(P.is_int[v] != 0, b.x, b.y)) {
            if (lane == 0) {
                key1[v] = -1;
                key2[v] = 0.0;
                key3[v] = INFINITY;
                flag[v] = 0;
            }
            continue;
        }
        const int cb = P.col_ptr[v], ce = P.col_ptr[v + 1];
        bool pos = false, neg = false;
        for (int s = cb + lane; s < ce; s += 32) {
            if (P.col_val[s] > 0) pos = true;
            else neg = true;
        }
        const bool mixed = __any_sync(0xffffffffu, pos) && __any_sync(0xffffffffu, neg);
        const double width = __dsub_rn(kdec(b.y), kdec(b.x));
        int cnt = 0;
        double exc = 0.0, unit = INFINITY;
        for (int s = cb + lane; s < ce; s += 32) {
            const int k = P.row_idx[s];
            const double gk = P.grow[k].x;
            if (ninf[k] != 0 || isinf(gk)) continue;
            const double a = fabs(P.col_val[s]);
            const double us = __ddiv_rn(__dsub_rn(gk, minfin[k]), a);
            unit = fmin(unit, us);
            if (mixed) {
                const double flipped = __dadd_rn(minfin[k], __dmul_rn(a, width));
                if (flipped > P.grow[k].y) {
                    ++cnt;
                    exc = fmax(exc, __dsub_rn(flipped, gk));
                }
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
            exc = fmax(exc, __shfl_xor_sync(0xffffffffu, exc, o));
            unit = fmin(unit, __shfl_xor_sync(0xffffffffu, unit, o));
        }
        if (lane == 0) {
            key1[v] = cnt;
            key2[v] = exc;
            key3[v] = unit;
            flag[v] = 1;
        }
    }
}

// radix key of a double: ascending order of the values (descending when `desc`)
__device__ __forceinline__ unsigned long long dbl_sort_key(double d, bool desc) {
    unsigned long long b = (unsigned long long)__double_as_longlong(d == 0.0 ? 0.0 : d);
    b = (b >> 63) ? ~b : (b | 0x8000000000000000ull);
    return desc ? ~b : b;
}

__global__ void k_keys_gather(int cnt, const int* idx, const int* key1, const double* key2, const double* key3,
                              int which, unsigned long long* keys) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += gridDim.x * blockDim.x) {
        const int v = idx[i];
        unsigned long long k;
        if (which == 3) k = dbl_sort_key(key3[v], false);
        else if (which == 2) k = dbl_sort_key(key2[v], true);
        else k = (unsigned long long)(0xffffffffu - (unsigned)key1[v]);   // key1 >= 0, descending
        keys[i] = k;
    }
}

__global__ void k_compact(int n, const int* flag, const int* pos, int* idx) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
        if (flag[v]) idx[pos[v]] = v;
}

static int grid_n(long long work) {
    long long b = (work + 255) / 256;
    return (int)(b < 1 ? 1 : (b > 1216 ? 1216 : b));
}

}  // namespace gpubp

using namespace gpubp;

extern "C" int bp_probe_priority(mip_problem* p, const double* lb, const double* ub, int32_t* key1, double* key2,
                                 double* key3, int32_t* order, int32_t* count, void* stream) {
    if (!p || !count || (p->n && (!lb || !ub || !key1 || !key2 || !key3 || !order))) {
        set_error("bp_probe_priority: null argument");
        return BP_ERR_INVALID;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const int n = p->n, m = p->m;
    *count = 0;
    if (n == 0) return BP_OK;
    longlong2* bk = p->w.bkey[0];
    double* minfin = nullptr;
    int *ninf = nullptr, *flag = nullptr, *pos = nullptr, *idx = nullptr, *tidx = nullptr, *total = nullptr;
    unsigned long long *keys = nullptr, *tkeys = nullptr;
    BP_CUDA_TRY(cudaMallocAsync(&minfin, sizeof(double) * (m ? m : 1), s));
    BP_CUDA_TRY(cudaMallocAsync(&ninf, sizeof(int) * (m ? m : 1), s));
    BP_CUDA_TRY(cudaMallocAsync(&flag, sizeof(int) * n, s));
    BP_CUDA_TRY(cudaMallocAsync(&pos, sizeof(int) * n, s));
    BP_CUDA_TRY(cudaMallocAsync(&idx, sizeof(int) * n, s));
    BP_CUDA_TRY(cudaMallocAsync(&tidx, sizeof(int) * n, s));
    BP_CUDA_TRY(cudaMallocAsync(&total, sizeof(int), s));
    BP_CUDA_TRY(cudaMallocAsync(&keys, sizeof(unsigned long long) * n, s));
    BP_CUDA_TRY(cudaMallocAsync(&tkeys, sizeof(unsigned long long) * n, s));
    int r = root_keys(p, lb, ub, bk, s);
    if (r != BP_OK) return r;
    if (m) k_row_minact<<<grid_n((long long)m * 32), 256, 0, s>>>(p->dp, bk, minfin, ninf);
    k_var_keys<<<grid_n((long long)n * 32), 256, 0, s>>>(p->dp, bk, minfin, ninf, key1, key2, key3, flag);
    BP_CUDA_TRY(cudaGetLastError());
    BP_TRY(scan_exclusive(flag, pos, n, total, s));
    k_compact<<<grid_n(n), 256, 0, s>>>(n, flag, pos, idx);
    int cnt = 0;
    BP_CUDA_TRY(cudaMemcpyAsync(&cnt, total, sizeof(int), cudaMemcpyDeviceToHost, s));
    BP_CUDA_TRY(cudaStreamSynchronize(s));
    if (cnt > 0) {
        // least significant key first: key3 ascending, then key2 descending, then key1 descending
        for (int which = 3; which >= 1; --which) {
            k_keys_gather<<<grid_n(cnt), 256, 0, s>>>(cnt, idx, key1, key2, key3, which, keys);
            BP_TRY(radix_sort_pairs(keys, idx, tkeys, tidx, cnt, 0, which == 1 ? 32 : 64, s));
        }
        BP_CUDA_TRY(cudaMemcpyAsync(order, idx, sizeof(int) * cnt, cudaMemcpyDeviceToDevice, s));
    }
    for (void* q : {(void*)minfin, (void*)ninf, (void*)flag, (void*)pos, (void*)idx, (void*)tidx, (void*)total,
                    (void*)keys, (void*)tkeys})
        BP_CUDA_TRY(cudaFreeAsync(q, s));
    BP_CUDA_TRY(cudaStreamSynchronize(s));
    *count = cnt;
    return BP_OK;
}
