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

}  // namespace gpubp
