// Learned rounding scorer: features, a 16-64-64-2 MLP on the fifth-generation tensor cores
// (BF16 operands, FP32 accumulators in tensor memory), its training step (loss gradient and
// Adam) and the scores that re-rank bulk fix-and-propagate (Section 2.3, Algorithm 1).
//
// The paper has no counterpart; propagation still judges every fixing the scorer proposes.
// Quantisation points (the oracle rounds at the same ones): features, hidden activations and
// the back-propagated pre-activation gradients are BF16; weights are FP32 masters rounded to
// BF16 for the products; biases, logits, the output-layer gradient and every accumulation are
// FP32.
//
// One CTA of 128 threads works on 128-row tiles; thread t owns row t of the tile and TMEM lane
// t.  Per tile: X -> [MMA] -> H1 -> [4 MMAs] -> H2 -> [4 MMAs] -> logits; in training also
// dZ3 -> dZ2 (CUDA cores: two outputs) -> [4 MMAs] dH1 -> dZ1, then one chain of 8 MMAs adds
// [dZ2 | dZ1]^T [H1 | X | 1] over the tile's rows into a TMEM accumulator that spans all the
// CTA's tiles: its blocks are dW2, dW1 and the bias gradients.  dW3 and db3 (two output units)
// are FP32 dot products over shared memory.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "bp_host.h"
#include "tc.cuh"

namespace gpubp {
namespace {

constexpr int kIn = 16, kHid = 64, kOut = 2;
constexpr int oW1 = 0, ob1 = oW1 + kHid * kIn, oW2 = ob1 + kHid, ob2 = oW2 + kHid * kHid, oW3 = ob2 + kHid,
              ob3 = oW3 + kOut * kHid, kNParam = ob3 + kOut;
static_assert(kNParam == 5378, "parameter count");
constexpr int kTile = 128;
constexpr int kMlpThreads = 128;
constexpr long long kWaitLimit = 2000000000LL;   // clock64 cycles (about 1 s) per MMA wait

// weight images (BF16, operand layout of tc.cuh), byte offsets
constexpr int kImgW1 = 0;                 // [64 out x 16 in]
constexpr int kImgW2 = 2048;              // [64 out x 64 in]
constexpr int kImgW3 = 10240;             // [16 out (2 used) x 64 in]
constexpr int kImgW2T = 12288;            // [64 in x 64 out]
constexpr int kImgBytes = 20480;

// shared memory of the forward kernel, byte offsets (1 KB aligned tiles).  H2 overwrites H1
// (layer 2 has read H1 by then) and the transposed W2 image of the backward pass is left out:
// 34 KB, so that six CTAs share an SM and their tiles' latency chains overlap.
constexpr int kSX = 0;                    // X tile       128 x 16
constexpr int kSH1 = kSX + 4096;          // H1, then H2  128 x 64
constexpr int kSW = kSH1 + 16384;         // weight images W1, W2, W3
constexpr int kImgFwdBytes = kImgW2T;     // the images the forward pass reads
constexpr int kSFloats = 64 + 64 + 4 + 128 + 256 + 4;   // b1[64] b2[64] b3[4] w3q[128] dz[256] red[4]
constexpr int kSFFwd = kSW + kImgFwdBytes;
constexpr int kSMiscFwd = kSFFwd + kSFloats * 4;        // mbarrier (8) and TMEM address (4)
constexpr int kSmemFwd = kSMiscFwd + 16;
// shared memory of the training kernel: tiles that are dead by the time another is written
// share space, so that two CTAs fit on an SM (110.7 KB each)
constexpr int kTH1 = 0;                   // H1 tile      128 x 64   (read by layer 2 only)
constexpr int kTDZ2 = kTH1;               // dZ2 tile     128 x 64   (written after layer 3)
constexpr int kTH2 = kTH1 + 16384;        // H2 tile      128 x 64
constexpr int kTW = kTH2 + 16384;         // weight images
constexpr int kTAW = kTW + kImgBytes;     // [dZ2 | dZ1]^T 128 x 128 (K = rows)
constexpr int kTX = kTAW;                 // X tile       128 x 16   (read by layer 1 only)
constexpr int kTBW = kTAW + 32768;        // [H1 | X | 1]^T 96 x 128
constexpr int kTF = kTBW + 24576;         // floats
constexpr int kTMisc = kTF + kSFloats * 4;
constexpr int kSmemTrain = kTMisc + 16;
constexpr int kTmemColsTrain = 256;       // 0..63: layer 1 / layer 3 / dH1, 64..127: layer 2, 128..223: weight grads
constexpr int kTmemColsFwd = 64;          // 0..63: layer 1, then layer 2, then layer 3 (each read out first)
constexpr int kTmemColsSM = 512;          // tensor memory columns of an SM

struct MlpArgs {
    const uint16_t* feat;     // rows x 16 BF16
    int rows;
    const unsigned char* wimg;
    const float* params;
    float* out;               // rows x 2 logits (forward)
    const float* labels;      // rows x 2, NaN = no label (training)
    const int* counts;        // labels per head (training)
    float* partial;           // gridDim.x x (kNParam + 1) (training)
    int* error;
};

__device__ __forceinline__ uint16_t* at16(unsigned char* base, uint32_t off) {
    return reinterpret_cast<uint16_t*>(base + off);
}

// All threads: bounded wait for the tile's MMAs, agreed by the whole CTA.
__device__ __forceinline__ bool wait_mma(uint32_t mbar, uint32_t& phase) {
    const bool ok = tc::mbar_wait(mbar, phase, kWaitLimit);
    phase ^= 1u;
    const int all = __syncthreads_and(ok ? 1 : 0);
    tc::fence_after_sync();
    return all != 0;
}

// Barrier between generic shared-memory writes and the next MMA (or TMEM reuse).
__device__ __forceinline__ void sync_for_mma() {
    tc::fence_smem_to_async();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
}

// 64 FP32 accumulator columns of this thread's lane -> bias, ReLU, BF16 into an A tile (row t,
// K = 64); returns the BF16 bits in hb.
__device__ __forceinline__ void hidden_from_tmem(uint32_t taddr, const float* bias, unsigned char* tile, int t,
                                                 uint16_t (&hb)[kHid]) {
#pragma unroll
    for (int c4 = 0; c4 < 4; ++c4) {
        float v[16];
        tc::tmem_ld16(taddr + 16 * c4, v);
#pragma unroll
        for (int j = 0; j < 16; j += 2) {
            // ReLU output is finite (fmaxf drops a NaN sum): the packed hardware conversion applies
            const uint32_t pk = tc::bf16x2_bits(fmaxf(v[j] + bias[16 * c4 + j], 0.0f),
                                                fmaxf(v[j + 1] + bias[16 * c4 + j + 1], 0.0f));
            hb[16 * c4 + j] = (uint16_t)pk;
            hb[16 * c4 + j + 1] = (uint16_t)(pk >> 16);
        }
    }
#pragma unroll
    for (int kc = 0; kc < 8; ++kc) {
        uint4 q;
        q.x = hb[8 * kc + 0] | ((uint32_t)hb[8 * kc + 1] << 16);
        q.y = hb[8 * kc + 2] | ((uint32_t)hb[8 * kc + 3] << 16);
        q.z = hb[8 * kc + 4] | ((uint32_t)hb[8 * kc + 5] << 16);
        q.w = hb[8 * kc + 6] | ((uint32_t)hb[8 * kc + 7] << 16);
        *reinterpret_cast<uint4*>(tile + tc::tile_off(t, 8 * kc, kHid)) = q;
    }
}

template <bool kTrain>
__global__ void __launch_bounds__(kMlpThreads, kTrain ? 2 : 6) k_mlp(MlpArgs a) {
    extern __shared__ __align__(1024) unsigned char sm[];
    const int t = threadIdx.x, warp = t >> 5;
    unsigned char* Xs = sm + (kTrain ? kTX : kSX);
    unsigned char* H1s = sm + (kTrain ? kTH1 : kSH1);
    unsigned char* H2s = sm + (kTrain ? kTH2 : kSH1);
    unsigned char* Ws = sm + (kTrain ? kTW : kSW);
    unsigned char* DZ2s = sm + kTDZ2;     // training only
    unsigned char* Aw = sm + kTAW;
    unsigned char* Bw = sm + kTBW;
    constexpr int kF = kTrain ? kTF : kSFFwd, kMisc = kTrain ? kTMisc : kSMiscFwd;
    constexpr uint32_t kTmemCols = kTrain ? kTmemColsTrain : kTmemColsFwd;
    constexpr uint32_t kL2 = kTrain ? 64 : 0;   // accumulator columns of layer 2
    float* b1 = reinterpret_cast<float*>(sm + kF);
    float* b2 = b1 + 64;
    float* b3 = b2 + 64;
    float* w3q = b3 + 4;
    float* dz = w3q + 128;
    float* red = dz + 256;
    uint64_t* mbar_p = reinterpret_cast<uint64_t*>(sm + kMisc);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(sm + kMisc + 8);
    const uint32_t mbar = tc::smem_u32(mbar_p);

    for (int i = t; i < (kTrain ? kImgBytes : kImgFwdBytes) / 16; i += kMlpThreads)
        reinterpret_cast<uint4*>(Ws)[i] = reinterpret_cast<const uint4*>(a.wimg)[i];
    if (t < kHid) {
        b1[t] = a.params[ob1 + t];
        b2[t] = a.params[ob2 + t];
    }
    if (t < 4) b3[t] = t < kOut ? a.params[ob3 + t] : 0.0f;
    for (int i = t; i < kOut * kHid; i += kMlpThreads) w3q[i] = tc::bf16_float(tc::bf16_bits(a.params[oW3 + i]));
    if (kTrain) {
        // rows 80..95 of [H1 | X | 1]^T: ones (their products give the bias gradients)
        for (int i = t; i < 16 * kTile; i += kMlpThreads)
            *at16(Bw, tc::tile_off(80 + i / kTile, i % kTile, kTile)) = 0x3f80;
    }
    if (t == 0) tc::mbar_init(mbar, 1);
    if (warp == 0) tc::tmem_alloc(tc::smem_u32(tmem_slot), kTmemCols);
    tc::fence_smem_to_async();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tm = *tmem_slot;
    const uint32_t lane = (uint32_t)(warp * 32) << 16;
    const uint32_t sW1 = tc::smem_u32(Ws + kImgW1), sW2 = tc::smem_u32(Ws + kImgW2),
                   sW3 = tc::smem_u32(Ws + kImgW3), sW2T = tc::smem_u32(Ws + kImgW2T);
    uint32_t phase = 0;
    bool ok = true;
    bool first = true;
    float acc_w3 = 0.0f, acc_b3 = 0.0f, loss = 0.0f;
    float inv_c0 = 0.0f, inv_c1 = 0.0f;
    if (kTrain) {
        inv_c0 = a.counts[0] > 0 ? 1.0f / (float)a.counts[0] : 0.0f;
        inv_c1 = a.counts[1] > 0 ? 1.0f / (float)a.counts[1] : 0.0f;
    }
    const int ntiles = (a.rows + kTile - 1) / kTile;
    // this thread's feature row of a tile (zero past the last row)
    auto load_row = [&](int tl, uint4& v0, uint4& v1) {
        const int r = tl * kTile + t;
        v0 = make_uint4(0, 0, 0, 0);
        v1 = make_uint4(0, 0, 0, 0);
        if (tl < ntiles && r < a.rows) {
            const uint4* src = reinterpret_cast<const uint4*>(a.feat + (size_t)r * kIn);
            v0 = src[0];
            v1 = src[1];
        }
    };
    // forward: the next tile's features are loaded while this tile's MMA chain runs
    uint4 nx0, nx1;
    if (!kTrain) load_row(blockIdx.x, nx0, nx1);
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int row = tile * kTile + t;
        const bool in = row < a.rows;
        // ---- features: X tile (A of layer 1) and, in training, rows 64..79 of [H1 | X | 1]^T
        uint4 x0, x1;
        if (kTrain) {
            load_row(tile, x0, x1);
        } else {
            x0 = nx0;
            x1 = nx1;
            load_row(tile + gridDim.x, nx0, nx1);
        }
        *reinterpret_cast<uint4*>(Xs + tc::tile_off(t, 0, kIn)) = x0;
        *reinterpret_cast<uint4*>(Xs + tc::tile_off(t, 8, kIn)) = x1;
        if (kTrain) {
            const uint32_t xw[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
#pragma unroll
            for (int i = 0; i < kIn; ++i)
                *at16(Bw, tc::tile_off(64 + i, t, kTile)) = (uint16_t)(xw[i >> 1] >> (16 * (i & 1)));
        }
        sync_for_mma();
        // ---- layer 1: D[0..63] = X W1^T
        if (t == 0) {
            tc::mma(tm + 0, tc::sdesc(tc::smem_u32(Xs), 128, 256), tc::sdesc(sW1, 128, 256), tc::idesc_bf16(128, 64), 0);
            tc::commit(mbar);
        }
        if (!(ok = wait_mma(mbar, phase))) break;
        uint16_t h1[kHid];
        hidden_from_tmem(tm + lane + 0, b1, H1s, t, h1);
        if (kTrain) {
#pragma unroll
            for (int i = 0; i < kHid; ++i) *at16(Bw, tc::tile_off(i, t, kTile)) = h1[i];
        }
        sync_for_mma();
        // ---- layer 2: D[64..127] = H1 W2^T
        if (t == 0) {
            for (int kk = 0; kk < 4; ++kk)
                tc::mma(tm + kL2, tc::sdesc(tc::smem_u32(H1s) + 256 * kk, 128, 1024), tc::sdesc(sW2 + 256 * kk, 128, 1024),
                        tc::idesc_bf16(128, 64), kk > 0);
            tc::commit(mbar);
        }
        if (!(ok = wait_mma(mbar, phase))) break;
        uint16_t h2[kHid];
        hidden_from_tmem(tm + lane + kL2, b2, H2s, t, h2);
        sync_for_mma();
        // ---- layer 3: D[0..15] = H2 W3^T (2 of 16 output columns used)
        if (t == 0) {
            for (int kk = 0; kk < 4; ++kk)
                tc::mma(tm + 0, tc::sdesc(tc::smem_u32(H2s) + 256 * kk, 128, 1024), tc::sdesc(sW3 + 256 * kk, 128, 1024),
                        tc::idesc_bf16(128, 16), kk > 0);
            tc::commit(mbar);
        }
        if (!(ok = wait_mma(mbar, phase))) break;
        float z[16];
        tc::tmem_ld16(tm + lane + 0, z);
        const float z0 = z[0] + b3[0], z1 = z[1] + b3[1];
        if (!kTrain) {
            if (in) {
                a.out[2 * (size_t)row] = z0;
                a.out[2 * (size_t)row + 1] = z1;
            }
        } else {
            // ---- loss gradient at the logits (per head: mean over its labels)
            float y0 = in ? a.labels[2 * (size_t)row] : NAN, y1 = in ? a.labels[2 * (size_t)row + 1] : NAN;
            float d0 = 0.0f, d1 = 0.0f;
            if (!isnan(y0)) {
                d0 = (1.0f / (1.0f + expf(-z0)) - y0) * inv_c0;
                loss += (fmaxf(z0, 0.0f) - z0 * y0 + log1pf(expf(-fabsf(z0)))) * inv_c0;
            }
            if (!isnan(y1)) {
                d1 = (1.0f / (1.0f + expf(-z1)) - y1) * inv_c1;
                loss += (fmaxf(z1, 0.0f) - z1 * y1 + log1pf(expf(-fabsf(z1)))) * inv_c1;
            }
            dz[t] = d0;
            dz[kTile + t] = d1;
            // dZ2 = (dZ3 W3q) * [H2 > 0] -> BF16: A of the dH1 product (row t) and rows 0..63 of
            // [dZ2 | dZ1]^T (column t)
            uint16_t g2[kHid];
#pragma unroll
            for (int i = 0; i < kHid; i += 2) {   // finite products: the packed conversion applies
                const uint32_t pk = tc::bf16x2_bits(d0 * w3q[i] + d1 * w3q[kHid + i],
                                                    d0 * w3q[i + 1] + d1 * w3q[kHid + i + 1]);
                g2[i] = h2[i] != 0 ? (uint16_t)pk : (uint16_t)0;
                g2[i + 1] = h2[i + 1] != 0 ? (uint16_t)(pk >> 16) : (uint16_t)0;
            }
#pragma unroll
            for (int kc = 0; kc < 8; ++kc) {
                uint4 q;
                q.x = g2[8 * kc + 0] | ((uint32_t)g2[8 * kc + 1] << 16);
                q.y = g2[8 * kc + 2] | ((uint32_t)g2[8 * kc + 3] << 16);
                q.z = g2[8 * kc + 4] | ((uint32_t)g2[8 * kc + 5] << 16);
                q.w = g2[8 * kc + 6] | ((uint32_t)g2[8 * kc + 7] << 16);
                *reinterpret_cast<uint4*>(DZ2s + tc::tile_off(t, 8 * kc, kHid)) = q;
            }
#pragma unroll
            for (int i = 0; i < kHid; ++i) *at16(Aw, tc::tile_off(i, t, kTile)) = g2[i];
            sync_for_mma();
            // dH1 = dZ2 W2q (B = W2^T image), into D[0..63]
            if (t == 0) {
                for (int kk = 0; kk < 4; ++kk)
                    tc::mma(tm + 0, tc::sdesc(tc::smem_u32(DZ2s) + 256 * kk, 128, 1024),
                            tc::sdesc(sW2T + 256 * kk, 128, 1024), tc::idesc_bf16(128, 64), kk > 0);
                tc::commit(mbar);
            }
            // meanwhile: dW3 and db3 of this tile, FP32 over shared memory in row order
            {
                const int o = t >> 6, i = t & 63;
                for (int b = 0; b < kTile; ++b)
                    acc_w3 += dz[o * kTile + b] * tc::bf16_float(*at16(H2s, tc::tile_off(b, i, kHid)));
                if (t < kOut)
                    for (int b = 0; b < kTile; ++b) acc_b3 += dz[t * kTile + b];
            }
            if (!(ok = wait_mma(mbar, phase))) break;
#pragma unroll
            for (int c4 = 0; c4 < 4; ++c4) {
                float v[16];
                tc::tmem_ld16(tm + lane + 16 * c4, v);
#pragma unroll
                for (int j = 0; j < 16; j += 2) {
                    const int i = 16 * c4 + j;
                    const uint32_t pk = tc::bf16x2_bits(v[j], v[j + 1]);
                    *at16(Aw, tc::tile_off(64 + i, t, kTile)) = h1[i] != 0 ? (uint16_t)pk : (uint16_t)0;
                    *at16(Aw, tc::tile_off(64 + i + 1, t, kTile)) = h1[i + 1] != 0 ? (uint16_t)(pk >> 16) : (uint16_t)0;
                }
            }
            sync_for_mma();
            // weight gradients: D[128..223] += [dZ2 | dZ1]^T [H1 | X | 1] over the tile's rows
            if (t == 0) {
                for (int kb = 0; kb < 8; ++kb)
                    tc::mma(tm + 128, tc::sdesc(tc::smem_u32(Aw) + 256 * kb, 128, 2048),
                            tc::sdesc(tc::smem_u32(Bw) + 256 * kb, 128, 2048), tc::idesc_bf16(128, 96),
                            (!first || kb > 0) ? 1u : 0u);
                tc::commit(mbar);
            }
            if (!(ok = wait_mma(mbar, phase))) break;
            first = false;
        }
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
    }
    if (kTrain && ok) {
        float* P = a.partial + (size_t)blockIdx.x * (kNParam + 1);
        if (first) {
            // no tile: zero weight-gradient blocks
            for (int i = t; i < kHid * kHid; i += kMlpThreads) P[oW2 + i] = 0.0f;
            for (int i = t; i < kHid * kIn; i += kMlpThreads) P[oW1 + i] = 0.0f;
            if (t < kHid) {
                P[ob2 + t] = 0.0f;
                P[ob1 + t] = 0.0f;
            }
        } else {
            // lanes 0..63: rows of dZ2^T (dW2 in columns 0..63, db2 in column 80); lanes 64..127:
            // rows of dZ1^T (dW1 in columns 64..79, db1 in column 80)
            const int o = t & 63;
            if (warp < 2) {
#pragma unroll
                for (int c4 = 0; c4 < 4; ++c4) {
                    float v[16];
                    tc::tmem_ld16(tm + lane + 128 + 16 * c4, v);
#pragma unroll
                    for (int j = 0; j < 16; ++j) P[oW2 + o * kHid + 16 * c4 + j] = v[j];
                }
                float v[16];
                tc::tmem_ld16(tm + lane + 128 + 80, v);
                P[ob2 + o] = v[0];
            } else {
                float v[16];
                tc::tmem_ld16(tm + lane + 128 + 64, v);
#pragma unroll
                for (int j = 0; j < 16; ++j) P[oW1 + o * kIn + j] = v[j];
                tc::tmem_ld16(tm + lane + 128 + 80, v);
                P[ob1 + o] = v[0];
            }
        }
        P[oW3 + t] = acc_w3;
        if (t < kOut) P[ob3 + t] = acc_b3;
        // loss: warp sums, then the four warps in order
        float s = loss;
        for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
        if ((t & 31) == 0) red[warp] = s;
        __syncthreads();
        if (t == 0) P[kNParam] = red[0] + red[1] + red[2] + red[3];
    }
    if (!ok && t == 0) atomicExch(a.error, BP_ERR_TIMEOUT);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 0) tc::tmem_free(tm, kTmemCols);
}

// BF16 images of the weights in the operand layout.
__global__ void k_weight_images(const float* params, unsigned char* img) {
    for (int i = threadIdx.x; i < kHid * kIn; i += blockDim.x) {
        const int o = i / kIn, k = i % kIn;
        *at16(img + kImgW1, tc::tile_off(o, k, kIn)) = tc::bf16_bits(params[oW1 + i]);
    }
    for (int i = threadIdx.x; i < kHid * kHid; i += blockDim.x) {
        const int o = i / kHid, k = i % kHid;
        const uint16_t w = tc::bf16_bits(params[oW2 + i]);
        *at16(img + kImgW2, tc::tile_off(o, k, kHid)) = w;
        *at16(img + kImgW2T, tc::tile_off(k, o, kHid)) = w;
    }
    for (int i = threadIdx.x; i < 16 * kHid; i += blockDim.x) {
        const int o = i / kHid, k = i % kHid;
        *at16(img + kImgW3, tc::tile_off(o, k, kHid)) = o < kOut ? tc::bf16_bits(params[oW3 + o * kHid + k]) : 0;
    }
}

// labels per head; launched with 256 threads and a few blocks per SM: one atomic per block
__global__ void k_label_counts(const float* labels, int rows, int* counts) {
    __shared__ int part[2][8];
    int c0 = 0, c1 = 0;
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < rows; r += gridDim.x * blockDim.x) {
        c0 += !isnan(labels[2 * (size_t)r]);
        c1 += !isnan(labels[2 * (size_t)r + 1]);
    }
    for (int off = 16; off > 0; off >>= 1) {
        c0 += __shfl_xor_sync(0xffffffffu, c0, off);
        c1 += __shfl_xor_sync(0xffffffffu, c1, off);
    }
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        part[0][w] = c0;
        part[1][w] = c1;
    }
    __syncthreads();
    if (threadIdx.x < 2) {
        int c = 0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) c += part[threadIdx.x][i];
        if (c) atomicAdd(counts + threadIdx.x, c);
    }
}

// gradient (and loss) = sum of the CTAs' partials, in CTA order
__global__ void k_grad_sum(const float* partial, int nparts, float* grad) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i <= kNParam; i += gridDim.x * blockDim.x) {
        float s = 0.0f;
        for (int c = 0; c < nparts; ++c) s += partial[(size_t)c * (kNParam + 1) + i];
        grad[i] = s;
    }
}

// Adam (Kingma and Ba, 2015), bias-corrected.
__global__ void k_adam(float* params, float* m, float* v, const float* grad, float lr, float b1, float b2, float eps,
                       float c1, float c2) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < kNParam; i += gridDim.x * blockDim.x) {
        const float g = grad[i];
        const float mi = b1 * m[i] + (1.0f - b1) * g;
        const float vi = b2 * v[i] + (1.0f - b2) * g * g;
        m[i] = mi;
        v[i] = vi;
        params[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

// ------------------------------------------------------------------------------ features
// BF16 of a double, round to nearest even (8 significant bits; below 2^-126 spacing 2^-133).
__device__ uint16_t bf16_from_double(double d) {
    if (isnan(d)) return 0x7fc0;
    if (d == 0.0 || isinf(d)) return (uint16_t)(__float_as_uint((float)d) >> 16);
    int e;
    frexp(d, &e);
    if (e < -125) e = -125;
    const double s = ldexp(1.0, 8 - e);
    const double r = rint(d * s) / s;
    if (fabs(r) >= 0x1p128) return d > 0 ? 0x7f80 : 0xff80;
    return (uint16_t)(__float_as_uint((float)r) >> 16);
}

// minimal activity of each row under raw bounds (finite part; infinite terms counted)
__global__ void k_feat_rows(DevProblem P, const double* lb, const double* ub, double* minfin, int* ninf) {
    const int lane = threadIdx.x & 31;
    for (int k = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; k < P.m; k += (gridDim.x * blockDim.x) >> 5) {
        double s = 0.0;
        int c = 0;
        for (int q = P.row_ptr[k] + lane; q < P.row_ptr[k + 1]; q += 32) {
            const double a = P.val[q];
            const double b = a > 0 ? lb[P.col[q]] : ub[P.col[q]];
            if (!(fabs(b) < kInfBound)) ++c;
            else s = __dadd_rn(s, __dmul_rn(a, b));
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

struct FeatCache {
    int npairs;
    const int* var;
    const int* status;
    const int64_t* offsets;
};

// raw features of vars[r] (warp per variable), FEATURES order of the oracle
__global__ void k_feat_vars(DevProblem P, const double* x, const double* lb, const double* ub, const double* obj,
                            const double* minfin, const int* ninf, const int* vars, int nvars, const int* pair_of,
                            FeatCache cache, double* raw) {
    const int lane = threadIdx.x & 31;
    for (int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < nvars; r += (gridDim.x * blockDim.x) >> 5) {
        const int j = vars[r];
        const int cb = P.col_ptr[j], ce = P.col_ptr[j + 1];
        double up = 0, dn = 0, absum = 0, S = 0;
        for (int q = cb + lane; q < ce; q += 32) {
            const double a = P.col_val[q];
            const int k = P.row_idx[q];
            up += a > 0;
            dn += a < 0;
            absum = __dadd_rn(absum, fabs(a));
            const double g = P.grow[k].x;
            if (ninf[k] == 0 && fabs(g) < kInfBound) {
                double sl = __dsub_rn(g, minfin[k]);
                if (sl < kTol) sl = kTol;
                const double t = __ddiv_rn(a, sl);
                S = __dadd_rn(S, __dmul_rn(t, t));
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            up += __shfl_xor_sync(0xffffffffu, up, o);
            dn += __shfl_xor_sync(0xffffffffu, dn, o);
            absum = __dadd_rn(absum, __shfl_xor_sync(0xffffffffu, absum, o));
            S = __dadd_rn(S, __shfl_xor_sync(0xffffffffu, S, o));
        }
        if (lane == 0) {
            const double deg = (double)(ce - cb);
            double rng = __dsub_rn(ub[j], lb[j]);
            if (!(rng <= 1e9)) rng = 1e9;
            const double fr = __dsub_rn(x[j], floor(x[j]));
            const double is_i = P.is_int[j] ? 1.0 : 0.0;
            double* f = raw + (size_t)r * 16;
            f[0] = deg;
            f[1] = log1p(deg);
            f[2] = obj ? obj[j] : 0.0;
            f[3] = up;
            f[4] = dn;
            f[5] = log1p(rng);
            f[6] = (is_i == 1.0 && rng <= 1.0) ? 1.0 : 0.0;
            f[7] = is_i;
            f[8] = fr;
            f[9] = fabs(__dsub_rn(fr, 0.5));
            f[10] = f[11] = f[12] = f[13] = 0.0;
            const int i = pair_of ? pair_of[j] : -1;
            if (i >= 0) {
                f[10] = (double)(cache.offsets[2 * i + 1] - cache.offsets[2 * i]);
                f[11] = (double)(cache.offsets[2 * i + 2] - cache.offsets[2 * i + 1]);
                f[12] = cache.status[2 * i] == 1 ? 1.0 : 0.0;
                f[13] = cache.status[2 * i + 1] == 1 ? 1.0 : 0.0;
            }
            f[14] = S;
            f[15] = absum;
        }
    }
}

// first pair of each probed variable
__global__ void k_pair_index(int npairs, const int* var, int* pair_of) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < npairs; i += gridDim.x * blockDim.x)
        atomicMin(pair_of + var[i], i);
}
__global__ void k_pair_none(int n, int npairs, int* pair_of) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x)
        if (pair_of[j] >= npairs) pair_of[j] = -1;
}

// per-feature mean and population standard deviation (block f; fixed reduction order)
__global__ void k_feat_stats(const double* raw, int nvars, double* stats) {
    __shared__ double red[256];
    const int f = blockIdx.x;
    double s = 0.0;
    for (int r = threadIdx.x; r < nvars; r += blockDim.x) s = __dadd_rn(s, raw[(size_t)r * 16 + f]);
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] = __dadd_rn(red[threadIdx.x], red[threadIdx.x + w]);
        __syncthreads();
    }
    const double mean = nvars > 0 ? red[0] / nvars : 0.0;
    __syncthreads();
    double q = 0.0;
    for (int r = threadIdx.x; r < nvars; r += blockDim.x) {
        const double d = __dsub_rn(raw[(size_t)r * 16 + f], mean);
        q = __dadd_rn(q, __dmul_rn(d, d));
    }
    red[threadIdx.x] = q;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] = __dadd_rn(red[threadIdx.x], red[threadIdx.x + w]);
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        double sd = nvars > 0 ? sqrt(red[0] / nvars) : 1.0;
        if (sd < 1e-12) sd = 1.0;
        stats[2 * f] = mean;
        stats[2 * f + 1] = sd;
    }
}

__global__ void k_feat_norm(const double* raw, int nvars, const double* stats, uint16_t* feat) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < (long long)nvars * 16;
         i += (long long)gridDim.x * blockDim.x) {
        const int f = (int)(i & 15);
        feat[i] = bf16_from_double(__ddiv_rn(__dsub_rn(raw[i], stats[2 * f]), stats[2 * f + 1]));
    }
}

__global__ void k_scores(const float* z, const int* vars, int rows, double* order_score, double* up_prob) {
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < rows; r += gridDim.x * blockDim.x) {
        const int j = vars[r];
        if (order_score) order_score[j] = (double)z[2 * (size_t)r];
        if (up_prob) up_prob[j] = 1.0 / (1.0 + exp(-(double)z[2 * (size_t)r + 1]));
    }
}

// labels of one feasible trajectory (see scorer_labels)
__global__ void k_labels(const double* x, const double* x_out, const int* vars, int nvars, float w, int first,
                         float* labels) {
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < nvars; r += gridDim.x * blockDim.x) {
        const int j = vars[r];
        const double xj = x[j], fixed = x_out[j];
        const double fl = floor(xj);
        float y0 = first ? 0.0f : labels[2 * (size_t)r];
        float y1 = first ? (xj == fl ? __int_as_float(0x7fc00000) : 0.0f) : labels[2 * (size_t)r + 1];
        if (fixed == floor(__dadd_rn(xj, 0.5))) y0 += w;
        if (fixed > xj) y1 += w;      // NaN stays NaN
        labels[2 * (size_t)r] = y0;
        labels[2 * (size_t)r + 1] = y1;
    }
}

int grid_for(long long work) {
    long long b = (work + 255) / 256;
    return (int)(b < 1 ? 1 : (b > 4096 ? 4096 : b));
}

}  // namespace
}  // namespace gpubp

using namespace gpubp;

struct scorer {
    int device = 0;
    int sms = 0;
    int fwd_per_sm = 1;        // resident forward CTAs per SM (shared memory and tensor memory bound)
    int train_per_sm = 1;      // resident training CTAs per SM
    float* params = nullptr;   // FP32 masters
    float* m = nullptr;
    float* v = nullptr;
    long long steps = 0;       // Adam steps taken
    unsigned char* wimg = nullptr;
    float* partial = nullptr;  // sms x train_per_sm x (kNParam + 1)
    float* grad = nullptr;     // kNParam + 1 (last: loss)
    int* counts = nullptr;
    int* error = nullptr;
};

namespace {

void scorer_release(scorer* s) {
    for (void* q : {(void*)s->params, (void*)s->m, (void*)s->v, (void*)s->wimg, (void*)s->partial, (void*)s->grad,
                    (void*)s->counts, (void*)s->error})
        if (q) cudaFree(q);
}

int refresh_images(scorer* s, cudaStream_t st) {
    k_weight_images<<<1, 256, 0, st>>>(s->params, s->wimg);
    BP_CUDA_TRY(cudaGetLastError());
    return BP_OK;
}

int check_error(scorer* s, cudaStream_t st) {
    int e = 0;
    BP_CUDA_TRY(cudaMemcpyAsync(&e, s->error, sizeof(int), cudaMemcpyDeviceToHost, st));
    BP_CUDA_TRY(cudaStreamSynchronize(st));
    if (e) {
        set_error("scorer: a tensor-core wait gave up");
        return BP_ERR_TIMEOUT;
    }
    return BP_OK;
}

// loss gradient of a batch into s->grad (and the loss into s->grad[kNParam])
int gradient(scorer* s, const uint16_t* feat, const float* labels, int rows, cudaStream_t st) {
    BP_CUDA_TRY(cudaMemsetAsync(s->counts, 0, 2 * sizeof(int), st));
    const int lb = (rows + 255) / 256;
    k_label_counts<<<lb < 4 * s->sms ? (lb > 0 ? lb : 1) : 4 * s->sms, 256, 0, st>>>(labels, rows, s->counts);
    MlpArgs a{feat, rows, s->wimg, s->params, nullptr, labels, s->counts, s->partial, s->error};
    const int ntiles = (rows + kTile - 1) / kTile;
    const int cap = s->sms * s->train_per_sm;
    const int grid = ntiles < cap ? (ntiles > 0 ? ntiles : 1) : cap;
    k_mlp<true><<<grid, kMlpThreads, kSmemTrain, st>>>(a);
    BP_CUDA_TRY(cudaGetLastError());
    k_grad_sum<<<grid_for(kNParam + 1), 256, 0, st>>>(s->partial, grid, s->grad);
    BP_CUDA_TRY(cudaGetLastError());
    return BP_OK;
}

}  // namespace

extern "C" int scorer_create(int32_t in, int32_t hidden, int32_t out, uint64_t seed, scorer** out_s) {
    if (!out_s || in != kIn || hidden != kHid || out != kOut) {
        set_error("scorer_create: only the 16-64-2 network is built (in=16, hidden=64, out=2)");
        return BP_ERR_INVALID;
    }
    *out_s = nullptr;
    scorer* s = new scorer();
    BP_CUDA_TRY(cudaGetDevice(&s->device));
    BP_CUDA_TRY(cudaDeviceGetAttribute(&s->sms, cudaDevAttrMultiProcessorCount, s->device));
    int smem_sm = 0;
    BP_CUDA_TRY(cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, s->device));
    // CTAs per SM: as many as shared memory (1 KB reserved per CTA) and tensor memory hold.  The
    // occupancy calculator reports 1 for these kernels, yet measured on GB300 several CTAs per SM
    // run faster.  Extra CTAs are safe whatever the residency: a CTA never waits on another, and
    // tcgen05.alloc only waits for columns that a running CTA frees at its end.
    s->fwd_per_sm = std::max(1, std::min(smem_sm / (kSmemFwd + 1024), kTmemColsSM / kTmemColsFwd));
    s->train_per_sm = std::max(1, std::min(smem_sm / (kSmemTrain + 1024), kTmemColsSM / kTmemColsTrain));
    bool okalloc = cudaMalloc(&s->params, sizeof(float) * kNParam) == cudaSuccess &&
                   cudaMalloc(&s->m, sizeof(float) * kNParam) == cudaSuccess &&
                   cudaMalloc(&s->v, sizeof(float) * kNParam) == cudaSuccess &&
                   cudaMalloc(&s->wimg, kImgBytes) == cudaSuccess &&
                   cudaMalloc(&s->partial, sizeof(float) * (size_t)s->sms * s->train_per_sm * (kNParam + 1)) ==
                       cudaSuccess &&
                   cudaMalloc(&s->grad, sizeof(float) * (kNParam + 1)) == cudaSuccess &&
                   cudaMalloc(&s->counts, 2 * sizeof(int)) == cudaSuccess &&
                   cudaMalloc(&s->error, sizeof(int)) == cudaSuccess;
    if (!okalloc) {
        scorer_release(s);
        delete s;
        set_error("scorer_create: out of device memory");
        return BP_ERR_OOM;
    }
    cudaError_t e = cudaFuncSetAttribute(k_mlp<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemTrain);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_mlp<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemFwd);
    // several CTAs share an SM only with a shared-memory carveout that holds them
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_mlp<false>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_mlp<true>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) {
        scorer_release(s);
        delete s;
        return fail_cuda(e, "cudaFuncSetAttribute");
    }
    // He-uniform weights, zero biases (splitmix64 chain, as the rounding draws)
    std::vector<float> h(kNParam, 0.0f);
    auto sm64 = [](uint64_t z) {
        z += 0x9E3779B97F4A7C15ull;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    };
    auto uni = [&](uint64_t a, uint64_t b, uint64_t c, uint64_t d) {
        uint64_t x = sm64(a);
        x = sm64(x ^ b);
        x = sm64(x ^ c);
        x = sm64(x ^ d);
        return (double)(x >> 11) * (1.0 / 9007199254740992.0);
    };
    const struct { int off, count, layer, fan_in; } mats[3] = {
        {oW1, kHid * kIn, 1, kIn}, {oW2, kHid * kHid, 2, kHid}, {oW3, kOut * kHid, 3, kHid}};
    for (const auto& M : mats) {
        const double lim = std::sqrt(6.0 / M.fan_in);
        for (int i = 0; i < M.count; ++i) h[M.off + i] = (float)((2.0 * uni(seed, 1000 + M.layer, i, 0) - 1.0) * lim);
    }
    *out_s = s;
    return scorer_set_params(s, h.data());
}

extern "C" void scorer_free(scorer* s) {
    if (!s) return;
    cudaDeviceSynchronize();
    scorer_release(s);
    delete s;
}

extern "C" int scorer_set_params(scorer* s, const float* host_params) {
    if (!s || !host_params) {
        set_error("scorer_set_params: null argument");
        return BP_ERR_INVALID;
    }
    BP_CUDA_TRY(cudaMemcpy(s->params, host_params, sizeof(float) * kNParam, cudaMemcpyHostToDevice));
    BP_CUDA_TRY(cudaMemset(s->m, 0, sizeof(float) * kNParam));
    BP_CUDA_TRY(cudaMemset(s->v, 0, sizeof(float) * kNParam));
    BP_CUDA_TRY(cudaMemset(s->error, 0, sizeof(int)));
    s->steps = 0;
    BP_TRY(refresh_images(s, nullptr));
    BP_CUDA_TRY(cudaDeviceSynchronize());
    return BP_OK;
}

extern "C" int scorer_get_params(const scorer* s, float* host_params) {
    if (!s || !host_params) {
        set_error("scorer_get_params: null argument");
        return BP_ERR_INVALID;
    }
    BP_CUDA_TRY(cudaDeviceSynchronize());
    BP_CUDA_TRY(cudaMemcpy(host_params, s->params, sizeof(float) * kNParam, cudaMemcpyDeviceToHost));
    return BP_OK;
}

extern "C" int scorer_forward(scorer* s, const uint16_t* feat, int32_t rows, float* out, void* stream) {
    if (!s || rows < 0 || (rows && (!feat || !out))) {
        set_error("scorer_forward: null or negative argument");
        return BP_ERR_INVALID;
    }
    if (rows == 0) return BP_OK;
    cudaStream_t st = (cudaStream_t)stream;
    MlpArgs a{feat, rows, s->wimg, s->params, out, nullptr, nullptr, nullptr, s->error};
    const int ntiles = (rows + kTile - 1) / kTile;
    const int cap = s->sms * s->fwd_per_sm;
    const int grid = ntiles < cap ? ntiles : cap;
    k_mlp<false><<<grid, kMlpThreads, kSmemFwd, st>>>(a);
    BP_CUDA_TRY(cudaGetLastError());
    return BP_OK;
}

extern "C" int scorer_scores(scorer* s, const uint16_t* feat, const int32_t* vars, int32_t rows, float* logits,
                             double* order_score, double* up_prob, void* stream) {
    if (!s || rows < 0 || (rows && (!vars || !logits))) {
        set_error("scorer_scores: null or negative argument");
        return BP_ERR_INVALID;
    }
    if (rows == 0) return BP_OK;
    BP_TRY(scorer_forward(s, feat, rows, logits, stream));
    k_scores<<<grid_for(rows), 256, 0, (cudaStream_t)stream>>>(logits, vars, rows, order_score, up_prob);
    BP_CUDA_TRY(cudaGetLastError());
    return BP_OK;
}

extern "C" int scorer_gradient(scorer* s, const uint16_t* feat, const float* labels, int32_t rows, float* grad_host,
                               float* loss_host, void* stream) {
    if (!s || rows <= 0 || !feat || !labels) {
        set_error("scorer_gradient: null argument or empty batch");
        return BP_ERR_INVALID;
    }
    cudaStream_t st = (cudaStream_t)stream;
    BP_TRY(gradient(s, feat, labels, rows, st));
    BP_TRY(check_error(s, st));
    if (grad_host) BP_CUDA_TRY(cudaMemcpyAsync(grad_host, s->grad, sizeof(float) * kNParam, cudaMemcpyDeviceToHost, st));
    if (loss_host) BP_CUDA_TRY(cudaMemcpyAsync(loss_host, s->grad + kNParam, sizeof(float), cudaMemcpyDeviceToHost, st));
    BP_CUDA_TRY(cudaStreamSynchronize(st));
    return BP_OK;
}

extern "C" int scorer_train_step(scorer* s, const uint16_t* feat, const float* labels, int32_t rows, float lr,
                                 float* loss_host, void* stream) {
    if (!s || rows <= 0 || !feat || !labels || !(lr > 0.0f)) {
        set_error("scorer_train_step: null argument, empty batch or lr <= 0");
        return BP_ERR_INVALID;
    }
    cudaStream_t st = (cudaStream_t)stream;
    BP_TRY(gradient(s, feat, labels, rows, st));
    s->steps += 1;
    const double b1 = 0.9, b2 = 0.999;
    const float c1 = (float)(1.0 - std::pow(b1, (double)s->steps)), c2 = (float)(1.0 - std::pow(b2, (double)s->steps));
    k_adam<<<grid_for(kNParam), 256, 0, st>>>(s->params, s->m, s->v, s->grad, lr, (float)b1, (float)b2, 1e-8f, c1, c2);
    BP_CUDA_TRY(cudaGetLastError());
    BP_TRY(refresh_images(s, st));
    if (loss_host) {
        BP_CUDA_TRY(cudaMemcpyAsync(loss_host, s->grad + kNParam, sizeof(float), cudaMemcpyDeviceToHost, st));
        BP_TRY(check_error(s, st));
    }
    return BP_OK;
}

extern "C" int scorer_features(mip_problem* p, const double* x, const double* lb, const double* ub,
                               const fp_cache* cache, const int32_t* vars, int32_t nvars, uint16_t* feat,
                               void* stream) {
    if (!p || nvars < 0 || (nvars && (!x || !lb || !ub || !vars || !feat))) {
        set_error("scorer_features: null or negative argument");
        return BP_ERR_INVALID;
    }
    if (nvars == 0) return BP_OK;
    cudaStream_t st = (cudaStream_t)stream;
    const int m = p->m, n = p->n;
    double *minfin = nullptr, *raw = nullptr, *stats = nullptr;
    int *ninf = nullptr, *pair_of = nullptr;
    BP_CUDA_TRY(cudaMallocAsync(&minfin, sizeof(double) * (m ? m : 1), st));
    BP_CUDA_TRY(cudaMallocAsync(&ninf, sizeof(int) * (m ? m : 1), st));
    BP_CUDA_TRY(cudaMallocAsync(&raw, sizeof(double) * 16 * (size_t)nvars, st));
    BP_CUDA_TRY(cudaMallocAsync(&stats, sizeof(double) * 32, st));
    FeatCache fc{0, nullptr, nullptr, nullptr};
    if (cache && cache->npairs > 0) {
        fc = FeatCache{cache->npairs, cache->var, cache->status, cache->offsets};
        BP_CUDA_TRY(cudaMallocAsync(&pair_of, sizeof(int) * (n ? n : 1), st));
        BP_CUDA_TRY(cudaMemsetAsync(pair_of, 0x7f, sizeof(int) * (n ? n : 1), st));
        k_pair_index<<<grid_for(cache->npairs), 256, 0, st>>>(cache->npairs, cache->var, pair_of);
        k_pair_none<<<grid_for(n), 256, 0, st>>>(n, cache->npairs, pair_of);
    }
    if (m) k_feat_rows<<<grid_for((long long)m * 32), 256, 0, st>>>(p->dp, lb, ub, minfin, ninf);
    k_feat_vars<<<grid_for((long long)nvars * 32), 256, 0, st>>>(p->dp, x, lb, ub, p->obj, minfin, ninf, vars, nvars,
                                                                pair_of, fc, raw);
    k_feat_stats<<<16, 256, 0, st>>>(raw, nvars, stats);
    k_feat_norm<<<grid_for((long long)nvars * 16), 256, 0, st>>>(raw, nvars, stats, feat);
    BP_CUDA_TRY(cudaGetLastError());
    for (void* q : {(void*)minfin, (void*)ninf, (void*)raw, (void*)stats, (void*)pair_of})
        if (q) BP_CUDA_TRY(cudaFreeAsync(q, st));
    return BP_OK;
}

extern "C" int scorer_labels(const double* x, const double* x_out, const int32_t* vars, int32_t nvars, float weight,
                             int32_t first, float* labels, void* stream) {
    if (nvars < 0 || (nvars && (!x || !x_out || !vars || !labels))) {
        set_error("scorer_labels: null or negative argument");
        return BP_ERR_INVALID;
    }
    if (nvars == 0) return BP_OK;
    k_labels<<<grid_for(nvars), 256, 0, (cudaStream_t)stream>>>(x, x_out, vars, nvars, weight, first ? 1 : 0, labels);
    BP_CUDA_TRY(cudaGetLastError());
    return BP_OK;
}

// File layout: magic "GPUBPML2", int32 {in, hidden, out, nparam}, int64 Adam steps, then the
// parameters, Adam's first and second moments (nparam floats each), little-endian.  Files of
// the first layout ("GPUBPML1": sizes and parameters only) still load, with a fresh Adam state.
extern "C" int scorer_save(const scorer* s, const char* path) {
    if (!s || !path) {
        set_error("scorer_save: null argument");
        return BP_ERR_INVALID;
    }
    std::vector<float> h(3 * (size_t)kNParam);
    BP_CUDA_TRY(cudaDeviceSynchronize());
    BP_CUDA_TRY(cudaMemcpy(h.data(), s->params, sizeof(float) * kNParam, cudaMemcpyDeviceToHost));
    BP_CUDA_TRY(cudaMemcpy(h.data() + kNParam, s->m, sizeof(float) * kNParam, cudaMemcpyDeviceToHost));
    BP_CUDA_TRY(cudaMemcpy(h.data() + 2 * kNParam, s->v, sizeof(float) * kNParam, cudaMemcpyDeviceToHost));
    FILE* f = fopen(path, "wb");
    if (!f) {
        set_error("scorer_save: cannot open %s", path);
        return BP_ERR_INVALID;
    }
    const char magic[8] = {'G', 'P', 'U', 'B', 'P', 'M', 'L', '2'};
    const int32_t dims[4] = {kIn, kHid, kOut, kNParam};
    const int64_t steps = s->steps;
    bool ok = fwrite(magic, 1, 8, f) == 8 && fwrite(dims, 4, 4, f) == 4 && fwrite(&steps, 8, 1, f) == 1 &&
              fwrite(h.data(), sizeof(float), h.size(), f) == h.size();
    ok = (fclose(f) == 0) && ok;
    if (!ok) {
        set_error("scorer_save: write to %s failed", path);
        return BP_ERR_INVALID;
    }
    return BP_OK;
}

extern "C" int scorer_load(scorer* s, const char* path) {
    if (!s || !path) {
        set_error("scorer_load: null argument");
        return BP_ERR_INVALID;
    }
    FILE* f = fopen(path, "rb");
    if (!f) {
        set_error("scorer_load: cannot open %s", path);
        return BP_ERR_INVALID;
    }
    char magic[8];
    int32_t dims[4];
    bool ok = fread(magic, 1, 8, f) == 8 && fread(dims, 4, 4, f) == 4;
    const bool v1 = ok && memcmp(magic, "GPUBPML1", 8) == 0;
    const bool v2 = ok && memcmp(magic, "GPUBPML2", 8) == 0;
    ok = ok && (v1 || v2) && dims[0] == kIn && dims[1] == kHid && dims[2] == kOut && dims[3] == kNParam;
    int64_t steps = 0;
    std::vector<float> h((v2 ? 3 : 1) * (size_t)kNParam);
    if (ok && v2) ok = fread(&steps, 8, 1, f) == 1 && steps >= 0;
    if (ok) ok = fread(h.data(), sizeof(float), h.size(), f) == h.size();
    fclose(f);
    if (!ok) {
        set_error("scorer_load: %s is not a 16-64-2 scorer file", path);
        return BP_ERR_INVALID;
    }
    BP_TRY(scorer_set_params(s, h.data()));   // parameters, fresh Adam state
    if (v2) {
        BP_CUDA_TRY(cudaMemcpy(s->m, h.data() + kNParam, sizeof(float) * kNParam, cudaMemcpyHostToDevice));
        BP_CUDA_TRY(cudaMemcpy(s->v, h.data() + 2 * kNParam, sizeof(float) * kNParam, cudaMemcpyHostToDevice));
        s->steps = steps;
    }
    return BP_OK;
}
