// Digit helpers shared by the split-digit tensor-core projections (the
// mma.sync kernels of ozaki.cu and the tcgen05 kernels of ozaki_tc.cu): the
// exponent field of a double, the balancing constant of the base-128 digits,
// and the recombination of the FP32 level sums into an FP64 value with
// integer operations.
#pragma once
#include <stdint.h>

namespace khp {
namespace oz {

constexpr int kS = 7;           // digits per value and levels kept

// exponent field of a double (0 for zero and subnormals, 2047 for Inf/NaN)
__device__ __forceinline__ int efield(double v) {
    return (int)((__double_as_longlong(v) >> 52) & 0x7ff);
}

// 64 in each of the six low base-128 digit positions: adding it turns the
// plain digits u_s of F into balanced ones, q_s = u_s - 64
constexpr unsigned long long kBal = 0x20408102040ull;

// v 2^sc for |v| < 2^52, built from the bit pattern (exact)
__device__ __forceinline__ double i2d_scaled(long long v, int sc) {
    if (v == 0) return 0.0;
    const unsigned long long sgn = v < 0 ? (1ull << 63) : 0ull;
    const unsigned long long a = (unsigned long long)(v < 0 ? -v : v);
    const int lz = __clzll((long long)a);
    const int e = 63 - lz;
    const unsigned long long mant = ((a << lz) << 1) >> 12;
    const int be = e + sc + 1023;
    if (be <= 0) return 0.0;
    if (be >= 2047) return __longlong_as_double((long long)(sgn | (0x7ffull << 52)));
    return __longlong_as_double((long long)(sgn | ((unsigned long long)be << 52) | mant));
}

// integer value of an FP32 holding an exact integer; SMALL: |c| < 2^22
// (magic-number conversion on the FMA/ALU pipes), else cvt
template <bool SMALL>
__device__ __forceinline__ long long f2ll(float c) {
    if (SMALL) return (long long)(__float_as_int(c + 12582912.0f) - 0x4B400000);
    return (long long)__float2int_rn(c);
}

// sum_L c[L] 2^(-7L) 2^(Ea + Eb - 14) with Ea = ea - 1022, Eb = eb - 1022
// (ea, eb exponent fields); NaN when either block held Inf/NaN
template <bool SMALL>
__device__ __forceinline__ double recombine(const float (&c)[kS], int ea, int eb) {
    if (ea == 2047 || eb == 2047) return __longlong_as_double(0x7ff8000000000000ll);
    long long hi = 0, lo = 0;
#pragma unroll
    for (int L = 0; L < 4; ++L) hi = hi * 128 + f2ll<SMALL>(c[L]);
#pragma unroll
    for (int L = 4; L < kS; ++L) lo = lo * 128 + f2ll<SMALL>(c[L]);
    const int E = (ea - 1022) + (eb - 1022) - 14;
    // sum_L c_L 2^-7L = hi 2^-21 + lo 2^-42
    return i2d_scaled(hi, E - 21) + i2d_scaled(lo, E - 42);
}

}  // namespace oz
}  // namespace khp
