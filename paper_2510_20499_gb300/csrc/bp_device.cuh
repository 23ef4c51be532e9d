// Device-side building blocks of the GB300 bound-propagation engine.
//
// Bounds live as interleaved pairs {l, u} (Section 2.1 keeps l_i, u_i at 2i, 2i+1 so that
// one gather fetches both) encoded as "ordered keys": an int64 whose signed order equals the
// numeric order of the double.  Tightening is then a plain atomicMin / atomicMax, and every
// comparison of bounds runs on the integer pipe: on GB300 each FP64 instruction (add, fma,
// compare, conversion, floor) issues at about 1/70 of the FP32 rate, so the hot loops spend
// exactly one FP64 instruction per nonzero (the fused multiply-add of the activity) and keep
// everything else in integer or FP32 arithmetic.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace gpubp {

constexpr double kTol = 1e-6;        // feasibility tolerance (Section 3)
constexpr double kInfBound = 1e20;   // |b| >= 1e20 means infinite
constexpr int kWarp = 32;

// ------------------------------------------------------------------ row classes
// Rows are binned by length (in the spirit of logarithmic radix binning, Section 2.1):
//   classes 0..3: at most 1, 2, 4, 8 nonzeros          -> one thread per row
//   class 4:      9 .. kWarpMax nonzeros               -> one warp per row
//   class 5:      (unused)
//   class 6:      more than kWarpMax nonzeros          -> "piece rows": pieces of chunk_len
//                                                         (kPieceMin .. kPieceMax) nonzeros, one
//                                                         warp each; a round sums the pieces'
//                                                         partial activities after a phase barrier
// Every task then holds at most kPerThread nonzeros per lane, all loaded in one wave, and all
// work of a round is warp-sized, so that it spreads over every SM of the grid.
constexpr int kNumClass = 7;
constexpr int kNumThreadBins = 4;
constexpr int kClassWarpRow = 4;
constexpr int kClassPieces = 6;
constexpr int kPerThread = 8;
constexpr int kThreadMax = kPerThread;            // 8
constexpr int kWarpMax = 32 * kPerThread;         // 256
constexpr int kPieceMax = kWarpMax;               // nonzeros of one piece: one wave of a warp
constexpr int kPieceMin = 32;                     // shortest piece length (sizes the piece lists)
// default split points (bp_autotune may pick others): a warp per row from 2 nonzeros, pieces
// for rows longer than kWarpMax, pieces of kDefaultChunkLen nonzeros
constexpr int kDefaultWarpMin = 2;
constexpr int kDefaultChunkLen = kPieceMax;

__host__ __device__ inline int row_class(int len) {
    if (len <= 1) return 0;
    if (len <= 2) return 1;
    if (len <= 4) return 2;
    if (len <= kThreadMax) return 3;
    if (len <= kWarpMax) return kClassWarpRow;
    return kClassPieces;
}

// Class of a row under tunable split points (the autotuner's search space): rows of block_min
// or more nonzeros are piece rows, rows of warp_min or more go to one warp, shorter rows to the
// thread bins above.  2 <= warp_min <= kThreadMax + 1 and warp_min <= block_min <= kWarpMax + 1;
// rows longer than kWarpMax are always piece rows.  warp_min = kThreadMax + 1,
// block_min = kWarpMax + 1 reproduce row_class.
__host__ __device__ inline int row_class_tuned(int len, int warp_min, int block_min) {
    if (len > kWarpMax || len >= block_min) return kClassPieces;
    if (len >= warp_min) return kClassWarpRow;
    return row_class(len);
}

// Piece descriptor {row, piece index c, first nonzero of the piece, end of the row}: the piece
// covers [beg, min(row end, beg + chunk_len)), the row has c + ceil((row end - beg) / chunk_len)
// pieces, and the row's pieces sit in consecutive slots of the round's piece list, c first-ones
// before this one, so no row data needs to be loaded to place or size the piece.
__host__ __device__ inline int4 piece_desc(int k, int c, int rb, int re, int len_c) {
    return make_int4(k, c, rb + c * len_c, re);
}

// ------------------------------------------------------------------ ordered keys
// key(d) = bits(d) for d >= +0, bits(d) ^ 0x7fff...f for negative d; -0.0 maps to +0.0 first
// so that the two zeros compare equal, as they do in IEEE arithmetic.
__device__ __forceinline__ long long dkey(double d) {
    long long b = __double_as_longlong(d);
    if (b == (long long)0x8000000000000000ULL) b = 0;
    return b >= 0 ? b : (b ^ 0x7fffffffffffffffLL);
}
__device__ __forceinline__ double kdec(long long k) {
    return __longlong_as_double(k >= 0 ? k : (k ^ 0x7fffffffffffffffLL));
}
__device__ __forceinline__ bool key_is_inf(long long k) {
    // +inf key = 0x7ff0...0; -inf key = 0xfff0...0 ^ 0x7fff...f = 0x800f...f
    return k == 0x7ff0000000000000LL || k == (long long)0x800fffffffffffffULL;
}
constexpr long long kKeyPosInf = 0x7ff0000000000000LL;
constexpr long long kKeyNegInf = (long long)0x800fffffffffffffULL;

// ------------------------------------------------------------ FP32 bracketing
// Directed conversions of a double to float by bit manipulation (integer pipe only):
// f_dn(x) <= x <= f_up(x).  They keep the 20 mantissa bits of the double's high word, so the
// truncation error is below one unit of the 20th bit (8 units of the float's last place);
// rounding up adds that unit.  The bracket is what the candidate prefilter needs, not accuracy.
__device__ __forceinline__ float mag_trunc(unsigned hi) {
    // |x| truncated toward zero, from the high word (sign cleared)
    unsigned mag = hi & 0x7fffffffu;
    if (mag >= 0x47f00000u) return mag >= 0x7ff00000u ? __int_as_float(0x7f800000) : 3.4028235e38f;
    if (mag < 0x38100000u) return 0.0f;
    return __int_as_float((int)((mag - 0x38000000u) << 3));
}
__device__ __forceinline__ float mag_round_up(unsigned hi) {
    unsigned mag = hi & 0x7fffffffu;
    if (mag >= 0x47f00000u) return __int_as_float(0x7f800000);
    if (mag < 0x38100000u) return mag == 0u ? 0.0f : 1.17549435e-38f;
    return __int_as_float((int)(((mag - 0x38000000u) << 3) + 8u));
}
__device__ __forceinline__ float f_up(double x) {
    unsigned hi = (unsigned)(__double_as_longlong(x) >> 32);
    unsigned lo = (unsigned)__double_as_longlong(x);
    if ((hi & 0x7fffffffu) == 0u && lo != 0u) return (int)hi < 0 ? 0.0f : 1.17549435e-38f;  // subnormal
    return (int)hi < 0 ? -mag_trunc(hi) : mag_round_up(hi);
}
__device__ __forceinline__ float f_dn(double x) {
    unsigned hi = (unsigned)(__double_as_longlong(x) >> 32);
    unsigned lo = (unsigned)__double_as_longlong(x);
    if ((hi & 0x7fffffffu) == 0u && lo != 0u) return (int)hi < 0 ? -1.17549435e-38f : 0.0f;
    return (int)hi < 0 ? -mag_round_up(hi) : mag_trunc(hi);
}
__device__ __forceinline__ float fabs_up(double x) {
    unsigned hi = (unsigned)(__double_as_longlong(x) >> 32);
    unsigned lo = (unsigned)__double_as_longlong(x);
    if ((hi & 0x7fffffffu) == 0u && lo != 0u) return 1.17549435e-38f;
    return mag_round_up(hi);
}

// ------------------------------------------------------------- memory helpers
__device__ __forceinline__ longlong2 ld_bounds(const longlong2* b, int j) {
    // bounds change during a launch: read through L2 (never a stale L1 line)
    return __ldcg(b + j);
}
__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ int ld_acquire_s32(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_u32(unsigned* p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void st_release_s32(int* p, int v) {
    asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned atom_add_acqrel_u32(unsigned* p, unsigned v) {
    unsigned old;
    asm volatile("atom.add.acq_rel.gpu.global.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}

// ----------------------------------------------------------- candidate math
// Candidate of variable j (coefficient a, round-start bounds {lk, uk}) from a row with
// finite activity part minfin and ninf infinite terms (Section 2.1):
//   a > 0: u <= (g - (minfin - a l)) / a,   a < 0: l >= (g - (minfin - a u)) / a
// (with ninf == 1 the variable is the infinite term and the residual is minfin itself), each
// operation rounded to nearest; integers round with floor(c + tol) / ceil(c - tol) and move
// on any improvement, continuous bounds move when the improvement exceeds
// theta * max(1, |old|) or the old bound is infinite.  Returns 1 (new upper key in *nk),
// 2 (new lower key in *nk) or 0 (nothing).
__device__ __forceinline__ int eval_candidate(double a, long long lk, long long uk, double minfin, int ninf,
                                              double g, bool is_i, double theta, long long* nk) {
    double resid;
    if (ninf == 1) {
        resid = minfin;
    } else {
        const double b = kdec(a > 0 ? lk : uk);
        resid = __dsub_rn(minfin, __dmul_rn(a, b));
    }
    const double num = __dsub_rn(g, resid);
    const double cand = __ddiv_rn(num, a);
    if (!(fabs(cand) < kInfBound)) return 0;
    if (a > 0) {
        if (is_i) {
            *nk = dkey(floor(__dadd_rn(cand, kTol)));
            return *nk < uk ? 1 : 0;
        }
        *nk = dkey(cand);
        if (uk == kKeyPosInf) return 1;
        const double u = kdec(uk);
        return __dsub_rn(u, cand) > __dmul_rn(theta, fmax(1.0, fabs(u))) ? 1 : 0;
    }
    if (is_i) {
        *nk = dkey(ceil(__dsub_rn(cand, kTol)));
        return *nk > lk ? 2 : 0;
    }
    *nk = dkey(cand);
    if (lk == kKeyNegInf) return 2;
    const double l = kdec(lk);
    return __dsub_rn(cand, l) > __dmul_rn(theta, fmax(1.0, fabs(l))) ? 2 : 0;
}

// Conservative test that a candidate from a row with finite activity cannot tighten the
// variable's bound: slack = g - L_min >= |a| (u - l) + margin, in FP32 with directed
// brackets.  The margin covers the rounding of the FP64 candidate (a few units of 2^-53 of
// |g| + |L_min| + |a| (|l| + |u|)), so a skipped candidate is one the exact evaluation would
// reject; a false "may tighten" only costs that evaluation.
struct RowFilter {
    float slack_dn;   // lower bracket of g - L_min (computed in FP64 once per row)
    float mag_up;     // upper bracket of |g| + |L_min|
};

__device__ __forceinline__ RowFilter row_filter(double g, double minfin) {
    RowFilter f;
    f.slack_dn = f_dn(__dsub_rn(g, minfin));
    f.mag_up = __fadd_ru(fabs_up(g), fabs_up(minfin));
    return f;
}

__device__ __forceinline__ bool cannot_tighten(const RowFilter& f, double a, long long lk, long long uk) {
    const double l = kdec(lk), u = kdec(uk);
    const float a_up = fabs_up(a);
    const float w_up = __fsub_ru(f_up(u), f_dn(l));
    const float prod = __fmul_ru(a_up, w_up);
    const float big = __fadd_ru(f.mag_up, __fmul_ru(2.0f, __fmul_ru(a_up, __fadd_ru(fabs_up(l), fabs_up(u)))));
    const float margin = __fmul_ru(1e-15f, big);
    return f.slack_dn >= __fadd_ru(prod, margin);
}

// Row infeasible: no infinite term and L_min > g + tol (gt = g + tol, precomputed).
__device__ __forceinline__ bool row_infeasible(double minfin, int ninf, double gt) {
    return ninf == 0 && dkey(minfin) > dkey(gt);
}

// Bounds cross: integer l > u, continuous l > u + tol.
__device__ __forceinline__ bool crossed(bool is_i, long long lk, long long uk) {
    if (lk <= uk) return false;
    if (is_i) return true;
    return kdec(lk) > __dadd_rn(kdec(uk), kTol);
}

// Normalised bound keys of a caller's (l, u): |b| >= 1e20 is infinite, integer bounds rounded
// inward with the tolerance.
__device__ __forceinline__ longlong2 normalized_keys(double l, double u, bool is_i) {
    if (l <= -kInfBound) l = -INFINITY;
    if (u >= kInfBound) u = INFINITY;
    if (is_i) {
        if (isfinite(l)) l = ceil(__dsub_rn(l, kTol));
        if (isfinite(u)) u = floor(__dadd_rn(u, kTol));
    }
    return make_longlong2(dkey(l), dkey(u));
}

// --------------------------------------------------------------- host structs
// Device view of a loaded problem.
struct DevProblem {
    int m, n, nnz;
    const int* row_ptr;          // m+1
    const int* col;              // nnz
    const double* val;           // nnz
    const double2* grow;         // m: {g, g + tol}, g = +inf for a free row
    const int* col_ptr;          // n+1 (transpose)
    const int* row_idx;          // nnz
    const double* col_val;       // nnz: coefficients in transpose order
    const unsigned char* is_int; // n
    const unsigned char* rclass; // m
    const int* rinfo;            // m: class | pieces << 3 (pieces of a piece row, else 0)
    const int* static_list;      // m: row ids grouped by class, ascending within a class
    const int4* static_tasks;    // every piece of the piece rows (round 0), see piece_desc
    int class_off[kNumClass + 1];// class segments of static_list and of worklists
    int chunk_len;               // nonzeros per piece of a piece row (kPieceMin .. kPieceMax)
    int nlong, npieces;          // piece rows, their pieces at chunk_len
};

}  // namespace gpubp
