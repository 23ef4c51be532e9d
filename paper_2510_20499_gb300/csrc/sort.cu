// Stable LSD radix sort of (uint64 key, int32 value) pairs on the device.
//
// Used for the probe priority order (Section 2.2) and the rounding orders of fix-and-propagate
// (Section 2.3, Algorithm 1): lexicographic orders are built from successive stable passes,
// least significant key first.  Each 8-bit digit pass: per-tile histograms, one exclusive scan
// over (digit, tile), then a stable scatter in which every tile ranks equal digits in input
// order (warp match for the rank inside a warp, shared-memory counts across warps and chunks).
// A pass whose digit is the same for every key is skipped.
#include "bp_host.h"

namespace gpubp {

constexpr int kSortThreads = 256;
constexpr int kSortTile = 4096;     // elements per tile (block)
constexpr int kRadix = 256;

__global__ void k_sort_hist(const unsigned long long* keys, int n, int shift, int* hist, int ntiles) {
    __shared__ int h[kRadix];
    for (int i = threadIdx.x; i < kRadix; i += blockDim.x) h[i] = 0;
    __syncthreads();
    const int t0 = blockIdx.x * kSortTile, t1 = min(n, t0 + kSortTile);
    for (int i = t0 + threadIdx.x; i < t1; i += blockDim.x) atomicAdd(&h[(keys[i] >> shift) & 0xff], 1);
    __syncthreads();
    for (int d = threadIdx.x; d < kRadix; d += blockDim.x) hist[d * ntiles + blockIdx.x] = h[d];
}

// digit totals: a digit holding all n keys means the pass would not move anything
__global__ void k_sort_digit_total(const int* hist, int ntiles, int n, int* uniform) {
    __shared__ int any_full;
    if (threadIdx.x == 0) any_full = 0;
    __syncthreads();
    for (int d = threadIdx.x; d < kRadix; d += blockDim.x) {
        int s = 0;
        for (int t = 0; t < ntiles; ++t) s += hist[d * ntiles + t];
        if (s == n) any_full = 1;
    }
    __syncthreads();
    if (threadIdx.x == 0) *uniform = any_full;
}

__global__ void k_sort_scatter(const unsigned long long* keys, const int* vals, int n, int shift, const int* offs,
                               int ntiles, const int* uniform, unsigned long long* okeys, int* ovals) {
    __shared__ int run[kRadix];                       // elements of each digit already placed by this tile
    __shared__ int wcnt[kSortThreads / 32][kRadix];   // per-warp digit counts of the current chunk
    const int w = threadIdx.x >> 5;
    const int t0 = blockIdx.x * kSortTile, t1 = min(n, t0 + kSortTile);
    if (*uniform) {   // nothing moves: copy
        for (int i = t0 + threadIdx.x; i < t1; i += blockDim.x) {
            okeys[i] = keys[i];
            ovals[i] = vals[i];
        }
        return;
    }
    for (int d = threadIdx.x; d < kRadix; d += blockDim.x) run[d] = 0;
    for (int base = t0; base < t1; base += blockDim.x) {
        for (int i = threadIdx.x; i < (kSortThreads / 32) * kRadix; i += blockDim.x) (&wcnt[0][0])[i] = 0;
        __syncthreads();
        const int i = base + threadIdx.x;
        const bool valid = i < t1;
        const unsigned long long k = valid ? keys[i] : 0ull;
        const int d = valid ? (int)((k >> shift) & 0xff) : -1;
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        unsigned lt;
        asm("mov.u32 %0, %%lanemask_lt;" : "=r"(lt));
        const int rank = __popc(peers & lt);
        if (valid && rank == 0) wcnt[w][d] = __popc(peers);
        __syncthreads();
        if (valid) {
            int before = run[d];
            for (int x = 0; x < w; ++x) before += wcnt[x][d];
            const int pos = offs[d * ntiles + blockIdx.x] + before + rank;
            okeys[pos] = k;
            ovals[pos] = vals[i];
        }
        __syncthreads();
        for (int dd = threadIdx.x; dd < kRadix; dd += blockDim.x) {
            int s = 0;
            for (int x = 0; x < kSortThreads / 32; ++x) s += wcnt[x][dd];
            run[dd] += s;
        }
        __syncthreads();
    }
}

// Sorts keys[0..n) with their values, stable, on bits [begin_bit, end_bit) (multiples of 8).
// tmp_keys / tmp_vals: n elements of scratch.  Result in keys / vals.
int radix_sort_pairs(unsigned long long* keys, int* vals, unsigned long long* tmp_keys, int* tmp_vals, int n,
                     int begin_bit, int end_bit, cudaStream_t s) {
    if (n <= 1) return BP_OK;
    const int ntiles = (n + kSortTile - 1) / kSortTile;
    int *hist = nullptr, *offs = nullptr, *uniform = nullptr;
    BP_CUDA_TRY(cudaMallocAsync(&hist, sizeof(int) * (size_t)kRadix * ntiles, s));
    BP_CUDA_TRY(cudaMallocAsync(&offs, sizeof(int) * (size_t)kRadix * ntiles, s));
    BP_CUDA_TRY(cudaMallocAsync(&uniform, sizeof(int), s));
    unsigned long long *ka = keys, *kb = tmp_keys;
    int *va = vals, *vb = tmp_vals;
    for (int shift = begin_bit; shift < end_bit; shift += 8) {
        k_sort_hist<<<ntiles, kSortThreads, 0, s>>>(ka, n, shift, hist, ntiles);
        k_sort_digit_total<<<1, kSortThreads, 0, s>>>(hist, ntiles, n, uniform);
        BP_TRY(scan_exclusive(hist, offs, kRadix * ntiles, nullptr, s));
        k_sort_scatter<<<ntiles, kSortThreads, 0, s>>>(ka, va, n, shift, offs, ntiles, uniform, kb, vb);
        BP_CUDA_TRY(cudaGetLastError());
        unsigned long long* tk = ka;
        ka = kb;
        kb = tk;
        int* tv = va;
        va = vb;
        vb = tv;
    }
    if (ka != keys) {
        BP_CUDA_TRY(cudaMemcpyAsync(keys, ka, sizeof(unsigned long long) * n, cudaMemcpyDeviceToDevice, s));
        BP_CUDA_TRY(cudaMemcpyAsync(vals, va, sizeof(int) * n, cudaMemcpyDeviceToDevice, s));
    }
    BP_CUDA_TRY(cudaFreeAsync(hist, s));
    BP_CUDA_TRY(cudaFreeAsync(offs, s));
    BP_CUDA_TRY(cudaFreeAsync(uniform, s));
    return BP_OK;
}

// ---------------------------------------------------------------- selection of the k smallest
// The first k entries of the stable sort of (key, value) pairs, without sorting the rest: an
// element's rank key is the 96-bit composite (key, position), unique, so the k smallest
// composites are exactly the stable sort's first k.  One block: a most-significant-digit radix
// select (12 digits of 8 bits: the key's 8 bytes, then the position's 4) finds the k-th smallest
// composite, the candidates sharing the prefix move to shared memory once few enough remain,
// then the k selected elements are gathered and sorted by their composite (bitonic network in
// shared memory).
constexpr int kSelThreads = 1024;

__device__ __forceinline__ int sel_digit(unsigned long long key, unsigned idx, int d) {
    return d < 8 ? (int)((key >> (56 - 8 * d)) & 0xff) : (int)((idx >> (24 - 8 * (d - 8))) & 0xff);
}

// -1, 0, 1: the composite's first `nd` digits below, equal to or above the prefix (pk, pi)
__device__ __forceinline__ int sel_cmp(unsigned long long key, unsigned idx, int nd, unsigned long long pk,
                                       unsigned pi) {
    if (nd <= 0) return 0;
    const int kb = nd < 8 ? nd : 8;
    const unsigned long long a = kb == 8 ? key : key >> (64 - 8 * kb), b = kb == 8 ? pk : pk >> (64 - 8 * kb);
    if (a != b) return a < b ? -1 : 1;
    if (nd <= 8) return 0;
    const int ib = nd - 8;
    const unsigned c = ib == 4 ? idx : idx >> (32 - 8 * ib), e = ib == 4 ? pi : pi >> (32 - 8 * ib);
    return c == e ? 0 : (c < e ? -1 : 1);
}

__global__ void __launch_bounds__(kSelThreads) k_select_smallest(const unsigned long long* keys, const int* vals,
                                                                 int n, int k, int* out) {
    __shared__ unsigned long long ck[kSelectMax];
    __shared__ unsigned ci[kSelectMax];
    __shared__ int hist[256];
    __shared__ int s_digit, s_kk, s_nc, s_pos;
    unsigned long long pk = 0;
    unsigned pi = 0;
    int kk = k;          // rank of the k-th smallest among the elements sharing the prefix
    bool shared_set = false;
    int nc = n;          // elements sharing the prefix
    int nd = 0;          // digits of the prefix
    while (nd < 12 && nc != kk) {
        for (int i = threadIdx.x; i < 256; i += kSelThreads) hist[i] = 0;
        __syncthreads();
        if (shared_set) {
            for (int i = threadIdx.x; i < nc; i += kSelThreads) atomicAdd(&hist[sel_digit(ck[i], ci[i], nd)], 1);
        } else {
            for (int i = threadIdx.x; i < n; i += kSelThreads) {
                const unsigned long long key = keys[i];
                if (sel_cmp(key, (unsigned)i, nd, pk, pi) == 0) atomicAdd(&hist[sel_digit(key, (unsigned)i, nd)], 1);
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            int below = 0, g = 0;
            while (below + hist[g] < kk) below += hist[g++];
            s_digit = g;
            s_kk = kk - below;
            s_nc = hist[g];
        }
        __syncthreads();
        const int g = s_digit;
        kk = s_kk;
        const int nc_new = s_nc;
        if (nd < 8) pk |= (unsigned long long)g << (56 - 8 * nd);
        else pi |= (unsigned)g << (24 - 8 * (nd - 8));
        ++nd;
        __syncthreads();
        if (shared_set) {
            // keep the candidates with the new digit (order does not matter: composites are unique)
            if (threadIdx.x == 0) s_pos = 0;
            __syncthreads();
            unsigned long long mk[(kSelectMax + kSelThreads - 1) / kSelThreads];
            unsigned mi[(kSelectMax + kSelThreads - 1) / kSelThreads];
            int mine = 0;
            for (int i = threadIdx.x; i < nc; i += kSelThreads)
                if (sel_digit(ck[i], ci[i], nd - 1) == g) {
                    mk[mine] = ck[i];
                    mi[mine] = ci[i];
                    ++mine;
                }
            __syncthreads();
            for (int q = 0; q < mine; ++q) {
                const int p = atomicAdd(&s_pos, 1);
                ck[p] = mk[q];
                ci[p] = mi[q];
            }
        } else if (nc_new <= kSelectMax) {
            if (threadIdx.x == 0) s_pos = 0;
            __syncthreads();
            for (int i = threadIdx.x; i < n; i += kSelThreads) {
                const unsigned long long key = keys[i];
                if (sel_cmp(key, (unsigned)i, nd, pk, pi) == 0) {
                    const int p = atomicAdd(&s_pos, 1);
                    ck[p] = key;
                    ci[p] = (unsigned)i;
                }
            }
            shared_set = true;
        }
        nc = nc_new;
        __syncthreads();
    }
    // the selected elements: first `nd` digits at or below the prefix (exactly k of them)
    if (threadIdx.x == 0) s_pos = 0;
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += kSelThreads) {
        const unsigned long long key = keys[i];
        if (sel_cmp(key, (unsigned)i, nd, pk, pi) <= 0) {
            const int p = atomicAdd(&s_pos, 1);
            if (p < kSelectMax) {
                ck[p] = key;
                ci[p] = (unsigned)i;
            }
        }
    }
    __syncthreads();
    int np2 = 1;
    while (np2 < k) np2 <<= 1;
    for (int i = k + threadIdx.x; i < np2; i += kSelThreads) {
        ck[i] = ~0ull;
        ci[i] = ~0u;
    }
    __syncthreads();
    // bitonic sort, ascending by (key, position)
    for (int size = 2; size <= np2; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = threadIdx.x; i < np2; i += kSelThreads) {
                const int j = i ^ stride;
                if (j > i) {
                    const bool up = (i & size) == 0;
                    const unsigned long long a = ck[i], b = ck[j];
                    const unsigned ia = ci[i], ib = ci[j];
                    const bool gt = a > b || (a == b && ia > ib);
                    if (gt == up) {
                        ck[i] = b;
                        ck[j] = a;
                        ci[i] = ib;
                        ci[j] = ia;
                    }
                }
            }
            __syncthreads();
        }
    }
    for (int i = threadIdx.x; i < k; i += kSelThreads) out[i] = vals[ci[i]];
}

// out[0..k) = the values of the first k pairs of the stable ascending sort of (keys, vals)[0..n),
// for 1 <= k <= min(n, kSelectMax); keys and vals are not modified.
int select_smallest(const unsigned long long* keys, const int* vals, int n, int k, int* out, cudaStream_t s) {
    if (k < 1 || k > n || k > kSelectMax) {
        set_error("select_smallest: k out of range");
        return BP_ERR_INVALID;
    }
    k_select_smallest<<<1, kSelThreads, 0, s>>>(keys, vals, n, k, out);
    BP_CUDA_TRY(cudaGetLastError());
    return BP_OK;
}

}  // namespace gpubp
