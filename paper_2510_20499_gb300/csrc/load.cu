// mip_load_csr: validation and device layouts of a MILP (Sections 1 and 2.1).
//
// Everything runs on the GPU: the row checks, the transpose (rows of each variable, needed
// to queue the rows of a changed variable), the length classes of the rows and the piece
// plan of long rows (pieces of one warp each).
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstring>

#include "bp_host.h"

namespace gpubp {

static thread_local std::string g_err;

void set_error(const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
}

int fail_cuda(cudaError_t e, const char* what) {
    set_error("CUDA error in %s: %s", what, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? BP_ERR_OOM : BP_ERR_CUDA;
}

// ------------------------------------------------------------------- scan
constexpr int kScanBlock = 1024;

__global__ void k_scan_block(const int* in, int* out, int n, int* block_sums) {
    __shared__ int s[kScanBlock];
    int i = blockIdx.x * kScanBlock + threadIdx.x;
    int v = i < n ? in[i] : 0;
    s[threadIdx.x] = v;
    __syncthreads();
    for (int off = 1; off < kScanBlock; off <<= 1) {
        int t = threadIdx.x >= off ? s[threadIdx.x - off] : 0;
        __syncthreads();
        s[threadIdx.x] += t;
        __syncthreads();
    }
    if (i < n) out[i] = s[threadIdx.x] - v;
    if (threadIdx.x == kScanBlock - 1) block_sums[blockIdx.x] = s[threadIdx.x];
}

__global__ void k_scan_add(int* out, int n, const int* block_offs) {
    int i = blockIdx.x * kScanBlock + threadIdx.x;
    if (i < n) out[i] += block_offs[blockIdx.x];
}

__global__ void k_scan_total(const int* in, const int* out, int n, int* total) {
    *total = n ? out[n - 1] + in[n - 1] : 0;
}

int scan_exclusive(const int* in, int* out, int n, int* total_dev, cudaStream_t s) {
    if (n <= 0) {
        if (total_dev) BP_CUDA_TRY(cudaMemsetAsync(total_dev, 0, sizeof(int), s));
        return BP_OK;
    }
    int nb = (n + kScanBlock - 1) / kScanBlock;
    int* sums = nullptr;
    int* offs = nullptr;
    BP_CUDA_TRY(cudaMallocAsync(&sums, sizeof(int) * nb, s));
    BP_CUDA_TRY(cudaMallocAsync(&offs, sizeof(int) * nb, s));
    k_scan_block<<<nb, kScanBlock, 0, s>>>(in, out, n, sums);
    if (nb > 1) {
        int r = scan_exclusive(sums, offs, nb, nullptr, s);
        if (r != BP_OK) return r;
        k_scan_add<<<nb, kScanBlock, 0, s>>>(out, n, offs);
    }
    if (total_dev) k_scan_total<<<1, 1, 0, s>>>(in, out, n, total_dev);
    BP_CUDA_TRY(cudaGetLastError());
    BP_CUDA_TRY(cudaFreeAsync(sums, s));
    BP_CUDA_TRY(cudaFreeAsync(offs, s));
    return BP_OK;
}

// ------------------------------------------------------------- validation
// error word: (index << 3) | code, smallest wins.  codes: 1 row_ptr, 2 column, 3 coefficient,
// 4 right-hand side, 5 bounds
__device__ __forceinline__ void report(unsigned long long* err, long long idx, int code) {
    atomicMin(err, ((unsigned long long)idx << 3) | (unsigned)code);
}

__global__ void k_validate_rows(int m, int n, long long nnz, const int64_t* rp, const int32_t* col,
                                const double* val, const double* g, unsigned long long* err) {
    // one warp per row
    const int lane = threadIdx.x & 31;
    for (long long k = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5; k < m;
         k += ((long long)gridDim.x * blockDim.x) >> 5) {
        const int64_t b = rp[k], e = rp[k + 1];
        // every access below stays inside [0, nnz): malformed offsets are reported, not read
        if (e < b || b < 0 || e > nnz) {
            if (lane == 0) report(err, k, 1);
            continue;
        }
        const double gk = g[k];
        if (lane == 0 && (isnan(gk) || gk <= -kInfBound)) report(err, k, 4);
        bool bad_col = false, bad_val = false;
        for (int64_t q = b + lane; q < e; q += 32) {
            const int j = col[q];
            if (j < 0 || j >= n || (q > b && j <= col[q - 1])) bad_col = true;
            const double a = val[q];
            if (!(fabs(a) >= 1e-12) || !(fabs(a) < kInfBound)) bad_val = true;
        }
        if (__any_sync(0xffffffffu, bad_col)) {
            if (lane == 0) report(err, k, 2);
        } else if (__any_sync(0xffffffffu, bad_val)) {
            if (lane == 0) report(err, k, 3);
        }
    }
}

__global__ void k_validate_bounds(int n, const double* lb, const double* ub, unsigned long long* err) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        double l = lb[j], u = ub[j];
        if (isnan(l) || isnan(u) || l >= kInfBound || u <= -kInfBound) report(err, j, 5);
    }
}

// ---------------------------------------------------------------- layouts
__global__ void k_rows(int m, const int64_t* rp64, const double* g, int* rp, double2* grow) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k <= m; k += gridDim.x * blockDim.x) {
        rp[k] = (int)rp64[k];
        if (k == m) continue;
        double gk = g[k] >= kInfBound ? (double)INFINITY : g[k];
        grow[k] = make_double2(gk, __dadd_rn(gk, kTol));
    }
}

// pieces of each piece row at piece length `len_c` (0 for other rows)
__global__ void k_row_pieces(int m, const int* rp, const unsigned char* rclass, int len_c, int* pieces) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < m; k += gridDim.x * blockDim.x)
        pieces[k] = rclass[k] == kClassPieces ? (rp[k + 1] - rp[k] + len_c - 1) / len_c : 0;
}

__global__ void k_reclass(int m, const int* rp, int warp_min, int block_min, int len_c, unsigned char* rclass,
                          int* rinfo) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < m; k += gridDim.x * blockDim.x) {
        const int len = rp[k + 1] - rp[k];
        const int c = row_class_tuned(len, warp_min, block_min);
        rclass[k] = (unsigned char)c;
        rinfo[k] = c | ((c == kClassPieces ? (len + len_c - 1) / len_c : 0) << 3);
    }
}

__global__ void k_class_flag(int m, const unsigned char* rclass, int c, int* flag) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < m; k += gridDim.x * blockDim.x)
        flag[k] = rclass[k] == c ? 1 : 0;
}

__global__ void k_class_scatter(int m, const unsigned char* rclass, int c, const int* pos, int base, int* list) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < m; k += gridDim.x * blockDim.x)
        if (rclass[k] == c) list[base + pos[k]] = k;
}

// every piece {row, piece} of the piece rows, rows ascending, pieces in row order
__global__ void k_piece_tasks(int m, const int* rp, const unsigned char* rclass, const int* pieces,
                              const int* piece_pos, int len_c, int4* tasks) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < m; k += gridDim.x * blockDim.x) {
        if (rclass[k] != kClassPieces) continue;
        const int base = piece_pos[k];
        for (int c = 0; c < pieces[k]; ++c) tasks[base + c] = piece_desc(k, c, rp[k], rp[k + 1], len_c);
    }
}

__global__ void k_col_count(long long nnz, const int32_t* col, int* cnt) {
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < nnz; q += (long long)gridDim.x * blockDim.x)
        atomicAdd(&cnt[col[q]], 1);
}

// transpose in a deterministic order: every column lists its rows ascending
__global__ void k_row_of(int m, const int* rp, int* row_of) {
    const int lane = threadIdx.x & 31;
    for (int k = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; k < m; k += (gridDim.x * blockDim.x) >> 5)
        for (int q = rp[k] + lane; q < rp[k + 1]; q += 32) row_of[q] = k;
}

__global__ void k_col_keys(long long nnz, const int32_t* col, unsigned long long* keys, int* pos) {
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < nnz; q += (long long)gridDim.x * blockDim.x) {
        keys[q] = (unsigned long long)col[q];
        pos[q] = (int)q;
    }
}

__global__ void k_col_fill(long long nnz, const int* pos, const int* row_of, const double* val, int* row_idx,
                           double* col_val) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nnz; i += (long long)gridDim.x * blockDim.x) {
        const int q = pos[i];
        row_idx[i] = row_of[q];
        col_val[i] = val[q];
    }
}

__global__ void k_norm_bounds(int n, const double* lb, const double* ub, const unsigned char* is_int,
                              double* ol, double* ou) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        double l = lb[j], u = ub[j];
        if (l <= -kInfBound) l = -INFINITY;
        if (u >= kInfBound) u = INFINITY;
        if (is_int[j]) {
            if (isfinite(l)) l = ceil(__dsub_rn(l, kTol));
            if (isfinite(u)) u = floor(__dadd_rn(u, kTol));
        }
        ol[j] = l;
        ou[j] = u;
    }
}

__global__ void k_is_int(int n, const uint8_t* in, unsigned char* out) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) out[j] = in[j] ? 1 : 0;
}

static int grid_for(long long work, int per_block = 256) {
    long long b = (work + per_block - 1) / per_block;
    if (b < 1) b = 1;
    if (b > 152 * 16) b = 152 * 16;
    return (int)b;
}

template <class T>
static int upload(mip_problem* p, const T* src, size_t count, int mem_kind, T** dst, cudaStream_t s) {
    BP_TRY(dalloc(p, dst, count));
    if (count)
        BP_CUDA_TRY(cudaMemcpyAsync(*dst, src, sizeof(T) * count,
                                    mem_kind == BP_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, s));
    return BP_OK;
}

// Row classes under the handle's split points, and the class-grouped static row list (each
// class ascending by row).
int classify_rows(mip_problem* p, cudaStream_t s) {
    DevProblem& dp = p->dp;
    const int m = p->m;
    int counts[kNumClass] = {};
    if (m) {
        unsigned char* rclass = const_cast<unsigned char*>(dp.rclass);
        int* list = const_cast<int*>(dp.static_list);
        k_reclass<<<grid_for(m), 256, 0, s>>>(m, dp.row_ptr, p->tune_warp_min, p->tune_block_min, dp.chunk_len,
                                              rclass, const_cast<int*>(dp.rinfo));
        BP_CUDA_TRY(cudaGetLastError());
        int *flag = nullptr, *pos = nullptr, *total = nullptr;
        BP_CUDA_TRY(cudaMallocAsync(&flag, sizeof(int) * ((size_t)m + 1), s));
        BP_CUDA_TRY(cudaMallocAsync(&pos, sizeof(int) * ((size_t)m + 1), s));
        BP_CUDA_TRY(cudaMallocAsync(&total, sizeof(int), s));
        int base = 0;
        for (int cl = 0; cl < kNumClass; ++cl) {
            k_class_flag<<<grid_for(m), 256, 0, s>>>(m, rclass, cl, flag);
            BP_TRY(scan_exclusive(flag, pos, m, total, s));
            k_class_scatter<<<grid_for(m), 256, 0, s>>>(m, rclass, cl, pos, base, list);
            BP_CUDA_TRY(cudaMemcpyAsync(&counts[cl], total, sizeof(int), cudaMemcpyDeviceToHost, s));
            BP_CUDA_TRY(cudaStreamSynchronize(s));
            base += counts[cl];
        }
        for (void* q : {(void*)flag, (void*)pos, (void*)total}) BP_CUDA_TRY(cudaFreeAsync(q, s));
    }
    int base = 0;
    for (int cl = 0; cl < kNumClass; ++cl) {
        dp.class_off[cl] = base;
        base += counts[cl];
    }
    dp.class_off[kNumClass] = base;
    dp.nlong = counts[kClassPieces];
    return BP_OK;
}

// Piece plan of the piece rows at the handle's piece length: every piece {row, piece}
// (static_tasks, the round-0 piece list).  The first call sizes the piece lists for the
// shortest piece length and any split point, so that later plans (bp_set_tuning) fit: a row of
// len nonzeros has at most len / kPieceMin + 1 pieces, so nnz / kPieceMin + m bound them all.
int plan_chunks(mip_problem* p, cudaStream_t s) {
    DevProblem& dp = p->dp;
    const int m = p->m;
    int rc = BP_OK;
    if (p->chunk_cap == 0) {
        const long long cap = (long long)dp.nnz / kPieceMin + (long long)m + 1;
        if (cap > INT_MAX) {
            set_error("piece lists of %lld entries exceed 32-bit indices", cap);
            return BP_ERR_CAPACITY;
        }
        p->chunk_cap = (int)cap;
        int4* tasks = nullptr;
        BP_TRY(dalloc(p, &tasks, (size_t)p->chunk_cap));
        dp.static_tasks = tasks;
    }
    dp.npieces = 0;
    if (!m) return BP_OK;
    int *pieces = nullptr, *pos = nullptr, *total = nullptr;
    const size_t words = (size_t)m + 1;
    BP_CUDA_TRY(cudaMallocAsync(&pieces, sizeof(int) * words, s));
    BP_CUDA_TRY(cudaMallocAsync(&pos, sizeof(int) * words, s));
    BP_CUDA_TRY(cudaMallocAsync(&total, sizeof(int), s));
    k_row_pieces<<<grid_for(m), 256, 0, s>>>(m, dp.row_ptr, dp.rclass, dp.chunk_len, pieces);
    if (cudaGetLastError() != cudaSuccess) rc = BP_ERR_CUDA;
    if (rc == BP_OK) rc = scan_exclusive(pieces, pos, m, total, s);
    int np = 0;
    if (rc == BP_OK && cudaMemcpyAsync(&np, total, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess) rc = BP_ERR_CUDA;
    if (rc == BP_OK && cudaStreamSynchronize(s) != cudaSuccess) rc = BP_ERR_CUDA;
    if (rc == BP_OK) {
        dp.npieces = np;
        k_piece_tasks<<<grid_for(m), 256, 0, s>>>(m, dp.row_ptr, dp.rclass, pieces, pos, dp.chunk_len,
                                                  const_cast<int4*>(dp.static_tasks));
        if (cudaGetLastError() != cudaSuccess) rc = BP_ERR_CUDA;
    }
    for (void* q : {(void*)pieces, (void*)pos, (void*)total}) cudaFreeAsync(q, s);
    BP_CUDA_TRY(cudaStreamSynchronize(s));
    if (rc == BP_ERR_CUDA) set_error("piece plan: CUDA error");
    return rc;
}

static int load_impl(int32_t m, int32_t n, const int64_t* row_ptr, const int32_t* col, const double* val,
                     const double* g, const double* lb, const double* ub, const uint8_t* is_int,
                     const double* c, int32_t mem_kind, cudaStream_t s, mip_problem* p) {
    if (m < 0 || n < 0) {
        set_error("negative dimensions m=%d n=%d", m, n);
        return BP_ERR_INVALID;
    }
    if (mem_kind != BP_MEM_HOST && mem_kind != BP_MEM_DEVICE) {
        set_error("mem_kind must be BP_MEM_HOST or BP_MEM_DEVICE");
        return BP_ERR_INVALID;
    }
    if (!row_ptr || (n && (!lb || !ub || !is_int)) || (m && !g)) {
        set_error("null array argument");
        return BP_ERR_INVALID;
    }
    BP_CUDA_TRY(cudaGetDevice(&p->device));
    // nnz and first-element check on the host (one 16-byte copy for device input)
    int64_t ends[2] = {0, 0};
    if (mem_kind == BP_MEM_HOST) {
        ends[0] = row_ptr[0];
        ends[1] = row_ptr[m];
    } else {
        BP_CUDA_TRY(cudaMemcpyAsync(&ends[0], row_ptr, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        BP_CUDA_TRY(cudaMemcpyAsync(&ends[1], row_ptr + m, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        BP_CUDA_TRY(cudaStreamSynchronize(s));
    }
    if (ends[0] != 0 || ends[1] < 0 || ends[1] >= (int64_t)INT32_MAX) {
        set_error("row_ptr[0] must be 0 and 0 <= nnz < 2^31 (got %lld, %lld)", (long long)ends[0],
                  (long long)ends[1]);
        return BP_ERR_INVALID;
    }
    if (ends[1] > 0 && (!col || !val)) {
        set_error("null col/val with nnz > 0");
        return BP_ERR_INVALID;
    }
    const int64_t nnz = ends[1];
    p->m = m;
    p->n = n;
    p->nnz = nnz;

    // raw copies on the device
    int64_t* d_rp64;
    int32_t* d_col;
    double *d_val, *d_g, *d_lb, *d_ub;
    uint8_t* d_isint_raw;
    BP_TRY(upload(p, row_ptr, (size_t)m + 1, mem_kind, &d_rp64, s));
    BP_TRY(upload(p, col, (size_t)nnz, mem_kind, &d_col, s));
    BP_TRY(upload(p, val, (size_t)nnz, mem_kind, &d_val, s));
    BP_TRY(upload(p, g, (size_t)m, mem_kind, &d_g, s));
    BP_TRY(upload(p, lb, (size_t)n, mem_kind, &d_lb, s));
    BP_TRY(upload(p, ub, (size_t)n, mem_kind, &d_ub, s));
    BP_TRY(upload(p, is_int, (size_t)n, mem_kind, &d_isint_raw, s));
    if (c) {
        BP_TRY(upload(p, c, (size_t)n, mem_kind, &p->obj, s));
    } else {
        BP_TRY(dalloc(p, &p->obj, (size_t)n));
    }

    // validation
    unsigned long long* d_err;
    BP_TRY(dalloc(p, &d_err, 1));
    BP_CUDA_TRY(cudaMemsetAsync(d_err, 0xff, sizeof(unsigned long long), s));
    if (m) k_validate_rows<<<grid_for((long long)m * 32), 256, 0, s>>>(m, n, nnz, d_rp64, d_col, d_val, d_g, d_err);
    if (n) k_validate_bounds<<<grid_for(n), 256, 0, s>>>(n, d_lb, d_ub, d_err);
    BP_CUDA_TRY(cudaGetLastError());
    unsigned long long herr = 0;
    BP_CUDA_TRY(cudaMemcpyAsync(&herr, d_err, sizeof(herr), cudaMemcpyDeviceToHost, s));
    BP_CUDA_TRY(cudaStreamSynchronize(s));
    if (herr != ~0ULL) {
        static const char* what[] = {"", "row_ptr not nondecreasing", "column out of range or not strictly increasing",
                                     "coefficient zero, tiny (<1e-12), infinite or NaN",
                                     "right-hand side NaN or -inf", "bound NaN, lb = +inf or ub = -inf"};
        int code = (int)(herr & 7);
        long long idx = (long long)(herr >> 3);
        set_error("invalid problem: %s at %s %lld", what[code < 6 ? code : 0], code == 5 ? "variable" : "row", idx);
        return BP_ERR_INVALID;
    }

    // row layouts
    DevProblem& dp = p->dp;
    dp.m = m;
    dp.n = n;
    dp.nnz = (int)nnz;
    int *d_rp, *d_list;
    double2* d_grow;
    unsigned char* d_rclass;
    BP_TRY(dalloc(p, &d_rp, (size_t)m + 1));
    BP_TRY(dalloc(p, &d_grow, (size_t)m));
    BP_TRY(dalloc(p, &d_rclass, (size_t)m));
    BP_TRY(dalloc(p, &d_list, (size_t)m));
    k_rows<<<grid_for(m + 1), 256, 0, s>>>(m, d_rp64, d_g, d_rp, d_grow);
    BP_CUDA_TRY(cudaGetLastError());
    int* d_rinfo;
    BP_TRY(dalloc(p, &d_rinfo, (size_t)m));
    dp.row_ptr = d_rp;
    dp.rclass = d_rclass;
    dp.rinfo = d_rinfo;
    dp.static_list = d_list;
    dp.chunk_len = kDefaultChunkLen;
    BP_TRY(classify_rows(p, s));
    // piece plan
    BP_TRY(plan_chunks(p, s));
    // transpose
    int *d_colcnt, *d_colptr, *d_fill, *d_rowidx;
    double* d_colval;
    BP_TRY(dalloc(p, &d_colval, (size_t)nnz));
    BP_TRY(dalloc(p, &d_colcnt, (size_t)n + 1));
    BP_TRY(dalloc(p, &d_colptr, (size_t)n + 1));
    BP_TRY(dalloc(p, &d_fill, (size_t)n + 1));
    BP_TRY(dalloc(p, &d_rowidx, (size_t)nnz));
    if (nnz) k_col_count<<<grid_for(nnz), 256, 0, s>>>(nnz, d_col, d_colcnt);
    BP_TRY(scan_exclusive(d_colcnt, d_colptr, n + 1, nullptr, s));
    if (nnz) {
        int *row_of = nullptr, *pos = nullptr, *tpos = nullptr;
        unsigned long long *keys = nullptr, *tkeys = nullptr;
        BP_CUDA_TRY(cudaMallocAsync(&row_of, sizeof(int) * nnz, s));
        BP_CUDA_TRY(cudaMallocAsync(&pos, sizeof(int) * nnz, s));
        BP_CUDA_TRY(cudaMallocAsync(&tpos, sizeof(int) * nnz, s));
        BP_CUDA_TRY(cudaMallocAsync(&keys, sizeof(unsigned long long) * nnz, s));
        BP_CUDA_TRY(cudaMallocAsync(&tkeys, sizeof(unsigned long long) * nnz, s));
        k_row_of<<<grid_for((long long)m * 32), 256, 0, s>>>(m, d_rp, row_of);
        k_col_keys<<<grid_for(nnz), 256, 0, s>>>(nnz, d_col, keys, pos);
        int bits = 8;
        while (bits < 32 && (1ll << bits) < (long long)n) bits += 8;
        BP_TRY(radix_sort_pairs(keys, pos, tkeys, tpos, (int)nnz, 0, bits, s));
        k_col_fill<<<grid_for(nnz), 256, 0, s>>>(nnz, pos, row_of, d_val, d_rowidx, d_colval);
        BP_CUDA_TRY(cudaGetLastError());
        for (void* q : {(void*)row_of, (void*)pos, (void*)tpos, (void*)keys, (void*)tkeys}) BP_CUDA_TRY(cudaFreeAsync(q, s));
    }
    // bounds and types
    unsigned char* d_isint;
    BP_TRY(dalloc(p, &d_isint, (size_t)n));
    BP_TRY(dalloc(p, &p->def_lb, (size_t)n));
    BP_TRY(dalloc(p, &p->def_ub, (size_t)n));
    if (n) {
        k_is_int<<<grid_for(n), 256, 0, s>>>(n, d_isint_raw, d_isint);
        k_norm_bounds<<<grid_for(n), 256, 0, s>>>(n, d_lb, d_ub, d_isint, p->def_lb, p->def_ub);
    }
    BP_CUDA_TRY(cudaGetLastError());
    dp.col = d_col;
    dp.val = d_val;
    dp.grow = d_grow;
    dp.col_ptr = d_colptr;
    dp.row_idx = d_rowidx;
    dp.col_val = d_colval;
    dp.is_int = d_isint;
    BP_TRY(engine_prepare(p));
    BP_CUDA_TRY(cudaStreamSynchronize(s));
    return BP_OK;
}

}  // namespace gpubp

using namespace gpubp;

extern "C" int mip_load_csr(int32_t m, int32_t n, const int64_t* row_ptr, const int32_t* col, const double* val,
                            const double* g, const double* lb, const double* ub, const uint8_t* is_int,
                            const double* c, int32_t mem_kind, void* stream, mip_problem** out) {
    if (!out) {
        set_error("out is null");
        return BP_ERR_INVALID;
    }
    *out = nullptr;
    mip_problem* p = new mip_problem();
    int r = load_impl(m, n, row_ptr, col, val, g, lb, ub, is_int, c, mem_kind, (cudaStream_t)stream, p);
    if (r != BP_OK) {
        cudaStreamSynchronize((cudaStream_t)stream);
        for (void* a : p->allocs) cudaFree(a);
        for (void* a : p->host_allocs) cudaFreeHost(a);
        delete p;
        return r;
    }
    *out = p;
    return BP_OK;
}

extern "C" int mip_free(mip_problem* p) {
    if (!p) return BP_OK;
    cudaDeviceSynchronize();
    for (auto hook : p->free_hooks)
        if (hook) hook(p);
    for (void* a : p->allocs) cudaFree(a);
    for (void* a : p->host_allocs) cudaFreeHost(a);
    delete p;
    return BP_OK;
}

extern "C" int mip_dims(const mip_problem* p, int32_t* m, int32_t* n, int64_t* nnz) {
    if (!p) {
        set_error("null handle");
        return BP_ERR_INVALID;
    }
    if (m) *m = p->m;
    if (n) *n = p->n;
    if (nnz) *nnz = p->nnz;
    return BP_OK;
}

extern "C" int mip_default_bounds(const mip_problem* p, double* lb, double* ub, void* stream) {
    if (!p || !lb || !ub) {
        set_error("null argument");
        return BP_ERR_INVALID;
    }
    cudaStream_t s = (cudaStream_t)stream;
    if (p->n) {
        BP_CUDA_TRY(cudaMemcpyAsync(lb, p->def_lb, sizeof(double) * p->n, cudaMemcpyDefault, s));
        BP_CUDA_TRY(cudaMemcpyAsync(ub, p->def_ub, sizeof(double) * p->n, cudaMemcpyDefault, s));
    }
    return BP_OK;
}

extern "C" const char* bp_last_error(void) { return g_err.c_str(); }

extern "C" const char* bp_version(void) { return "gpubp 0.1 (sm_103a)"; }

extern "C" void bp_params_default(bp_params* p) {
    if (!p) return;
    p->theta = 1e-3;
    p->max_rounds = 10000;
    p->bounds_mem = BP_MEM_DEVICE;
    p->trace = nullptr;
}

extern "C" int probe_split(int32_t is_int, double l, double u, double* box4) {
    if (!is_int || !(l < u) || !box4) return 0;
    if (std::isfinite(l) && std::isfinite(u)) {
        double c = std::ceil((l + u) / 2.0);
        box4[0] = l;
        box4[1] = c - 1.0;
        box4[2] = c;
        box4[3] = u;
        return 1;
    }
    if (std::isfinite(l)) {
        box4[0] = l;
        box4[1] = l;
        box4[2] = l + 1.0;
        box4[3] = INFINITY;
        return 1;
    }
    if (std::isfinite(u)) {
        box4[0] = u;
        box4[1] = u;
        box4[2] = -INFINITY;
        box4[3] = u - 1.0;
        return 1;
    }
    return 0;
}
