// Counter-based draws and the rounding distribution of fix-and-propagate (Section 2.3).
//
// uniform01: splitmix64 chained over (seed, bulk, variable, draw), the top 53 bits as a double in
// [0, 1).  draw_value: the rounding of x in the paper's distribution (fractional part f <= 0.25
// rounds down, f >= 0.75 rounds up, in between up with probability (f - 0.25) / 0.5, or with a
// given per-variable up probability).
#pragma once

namespace gpubp {

__device__ __forceinline__ unsigned long long sm64(unsigned long long z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ double uniform01(unsigned long long seed, unsigned long long bulk, unsigned long long var,
                                            unsigned long long draw) {
    unsigned long long h = sm64(seed);
    h = sm64(h ^ bulk);
    h = sm64(h ^ var);
    h = sm64(h ^ draw);
    return __dmul_rn(__ull2double_rn(h >> 11), 1.0 / 9007199254740992.0);
}

__device__ __forceinline__ double clampd(double x, double l, double u) { return x < l ? l : (x > u ? u : x); }

__device__ __forceinline__ double draw_value(double x, unsigned long long seed, unsigned long long bulk, int j, int d,
                                             const double* up_prob) {
    const double fl = floor(x);
    const double f = __dsub_rn(x, fl);
    if (f == 0.0) return x;
    double pup;
    if (f <= 0.25) pup = 0.0;
    else if (f >= 0.75) pup = 1.0;
    else pup = up_prob ? up_prob[j] : __ddiv_rn(__dsub_rn(f, 0.25), 0.5);
    return uniform01(seed, bulk, (unsigned long long)j, (unsigned long long)d) < pup ? __dadd_rn(fl, 1.0) : fl;
}

}  // namespace gpubp
