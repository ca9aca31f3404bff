// Rayleigh-Ritz projections on the tensor cores with FP64 accuracy.
//
// The two dense contractions of every outer iteration (Sec. II B) are the
// Gram matrices G = Y^H Y, S = Y^H (H Y) (a reduction over the 2.2M-long grid
// dimension) and the rotation [X, HX] = [Y, HY] Q.  On B300 the FP64 ALUs
// run at 1/64 of the FP32 rate, so both are computed here as exact integer
// products on the BF16 tensor cores (mma.sync m16n8k16, FP32 accumulate):
//
//  * every FP64 value v of a block that shares the exponent bound 2^E
//    (a column of a 64-row chunk for the Gram, a row for the rotation, a
//    column of Q) is rounded to 49 bits below the bound and cut into seven
//    balanced base-128 digits,
//        v ~= sum_{s<7} d_s 2^(E - 7(s+1)),  |d_s| <= 64 (s >= 1), |d_0| <= 128,
//    (the digits come from the bit pattern by integer operations; each
//    digit is exact in BF16);
//  * digit blocks are multiplied pairwise on the tensor cores; products with
//    the same level L = s + t share one scale and are summed in one FP32
//    accumulator.  With K <= 64 terms and at most 7 pairs per level every
//    partial sum is an integer below 2^22, so the FP32 accumulation is exact;
//  * levels L <= 6 are kept (28 digit pairs); the dropped products are of
//    order 2^-49 of sum |a_k b_k| with random signs, below the rounding of
//    an FP64 evaluation of the same sum;
//  * the seven level sums are recombined in int64 and turned into FP64
//    with integer operations, so the FP64 pipe only adds the results.
//
// This is the splitting scheme of Ozaki et al. (error-free matrix
// multiplication by splitting into low-precision slices) written for
// BF16 digits and exact FP32 accumulation.
#include <math.h>
#include <stdint.h>

#include <algorithm>

#include "khp_common.cuh"
#include "khp_internal.h"

namespace khp {
namespace oz {

constexpr int kS = 7;           // digits per value and levels kept
constexpr int kMaxM = 32;       // complex columns (real width 64)
constexpr int kChunk = 64;      // Gram rows per exponent block
constexpr int kTile = 64;       // rotation rows per tile
constexpr int kGramWarps = 12;
constexpr int kRotWarps = 8;

__host__ __device__ constexpr int round16(int v) { return (v + 15) & ~15; }

// exponent field of a double (0 for zero and subnormals, 2047 for Inf/NaN)
__device__ __forceinline__ int efield(double v) {
    return (int)((__double_as_longlong(v) >> 52) & 0x7ff);
}

// BF16 bit pattern of a digit of magnitude q <= 128 (exact), sign in bit 15
__device__ __forceinline__ uint32_t bf16_digit(uint32_t q, uint32_t sgn) {
    const float f = __uint_as_float(0x4B000000u | q) - 8388608.0f;
    return q ? ((__float_as_uint(f) >> 16) | sgn) : 0u;
}

// digits of v against the block's exponent field emax (|v| < 2^(emax-1022)):
// F = round(|v| 2^(49-E)) <= 2^49, written in balanced base 128,
// F = sum_s q_s 128^(6-s) with |q_s| <= 64 for s >= 1 and 0 <= q_0 <= 128;
// the digits carry the sign of v.  Balanced digits make the dropped
// low-level products of a value with itself (the Gram diagonal) average out.
__device__ __forceinline__ void split(double v, int emax, uint16_t (&d)[kS]) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    const int ex = (int)((b >> 52) & 0x7ff);
    const uint32_t sgn = (uint32_t)(b >> 48) & 0x8000u;
    unsigned long long F = 0;
    if (ex != 0 && emax < 2047) {
        const unsigned long long mant = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
        const int sh = emax - ex + 4;          // >= 4
        if (sh < 64) F = (mant >> sh) + ((mant >> (sh - 1)) & 1ull);
    }
    int q[kS];
#pragma unroll
    for (int s = kS - 1; s >= 1; --s) {
        int r = (int)(F & 127ull);
        F >>= 7;
        if (r >= 64) {
            r -= 128;
            F += 1;
        }
        q[s] = r;
    }
    q[0] = (int)F;
#pragma unroll
    for (int s = 0; s < kS; ++s) {
        const uint32_t a = (uint32_t)(q[s] < 0 ? -q[s] : q[s]);
        d[s] = (uint16_t)bf16_digit(a, q[s] < 0 ? (sgn ^ 0x8000u) : sgn);
    }
}

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

// sum_L c[L] 2^(-7L) 2^(Ea + Eb - 14) with Ea = ea - 1022, Eb = eb - 1022
// (ea, eb exponent fields); NaN when either block held Inf/NaN
__device__ __forceinline__ double recombine(const float (&c)[kS], int ea, int eb) {
    if (ea == 2047 || eb == 2047) return __longlong_as_double(0x7ff8000000000000ll);
    long long hi = 0, lo = 0;
#pragma unroll
    for (int L = 0; L < 4; ++L) hi = hi * 128 + (long long)__float2int_rn(c[L]);
#pragma unroll
    for (int L = 4; L < kS; ++L) lo = lo * 128 + (long long)__float2int_rn(c[L]);
    const int E = (ea - 1022) + (eb - 1022) - 14;
    // sum_L c_L 2^-7L = hi 2^-21 + lo 2^-42
    return i2d_scaled(hi, E - 21) + i2d_scaled(lo, E - 42);
}

__device__ __forceinline__ void mma(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
        "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ uint32_t ld32(const uint16_t* p) { return *reinterpret_cast<const uint32_t*>(p); }

// ------------------------------------------------------------------ Gram
// A = [Re Y | Im Y] (rows x 2m), B = [Re W | Im W]; per CTA and chunk of 64
// rows: digits of A^T and B^T in shared memory ([slice][column][row], rows
// contiguous, padded), D_G += A^T A and D_S += A^T B over the CTA's rows
// (FP64 in shared memory), then the packed upper triangles of the complex
// G_ij = D[i][j] + D[i+m][j+m] + i (D[i][j+m] - D[i+m][j]) (and S) as the
// CTA's partial.  Warp unit = (matrix, 16-row m-tile, group of 3 n-tiles).
constexpr int kRowStride = kChunk + 8;   // padded digit row (bank-conflict free fragments)

struct GramSmem {
    static size_t bytes(int m, bool w) {
        const int RP = round16(2 * m);
        const size_t dig = (size_t)(w ? 2 : 1) * kS * RP * kRowStride * sizeof(uint16_t);
        const size_t acc = (size_t)(w ? 2 : 1) * RP * RP * sizeof(double);
        return dig + acc + 2 * RP * sizeof(int) * 2;
    }
};

__global__ void __launch_bounds__(kGramWarps * 32, 1)
    gram_oz_kernel(const double2* __restrict__ Y, const double2* __restrict__ W, long long rows, int ld, int col0,
                   int m, double2* __restrict__ partial) {
    extern __shared__ __align__(16) unsigned char sm[];
    const bool hasW = W != nullptr;
    const int nmat = hasW ? 2 : 1;
    const int R2 = 2 * m, RP = round16(R2);
    uint16_t* Ad = reinterpret_cast<uint16_t*>(sm);                  // [kS][RP][kRowStride]
    uint16_t* Bd = Ad + (size_t)kS * RP * kRowStride;                // same, W (if any)
    double* D = reinterpret_cast<double*>(Bd + (hasW ? (size_t)kS * RP * kRowStride : 0));  // [nmat][RP][RP]
    int* ea = reinterpret_cast<int*>(D + (size_t)nmat * RP * RP);    // [RP] chunk column exponents of A
    int* eb = ea + RP;                                               // [RP] of B
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nthr = blockDim.x;

    for (int i = tid; i < nmat * RP * RP; i += nthr) D[i] = 0.0;
    // padding columns (real index >= 2m) keep zero digits for the whole run
    for (int i = tid; i < (hasW ? 2 : 1) * kS * RP * kRowStride; i += nthr) Ad[i] = 0;

    const long long nchunks = (rows + kChunk - 1) / kChunk;
    const long long per = (nchunks + gridDim.x - 1) / gridDim.x;
    const long long c0 = (long long)blockIdx.x * per;
    const long long c1 = c0 + per < nchunks ? c0 + per : nchunks;

    const int MT = RP / 16, NT = RP / 8, NG = (NT + 2) / 3;
    const int units = nmat * MT * NG;
    const int g = lane >> 2, tg = lane & 3;

    for (long long ch = c0; ch < c1; ++ch) {
        const long long r0 = ch * kChunk;
        const int nr = (int)(rows - r0 < kChunk ? rows - r0 : kChunk);
        __syncthreads();   // previous chunk's fragments are consumed
        for (int i = tid; i < 2 * RP; i += nthr) ea[i] = 0;
        __syncthreads();
        // column exponent bounds of this chunk
        for (int idx = tid; idx < kChunk * m; idx += nthr) {
            const int r = idx / m, c = idx - r * m;
            if (r < nr) {
                const double2 y = Y[(r0 + r) * ld + col0 + c];
                atomicMax(&ea[c], efield(y.x));
                atomicMax(&ea[c + m], efield(y.y));
                if (hasW) {
                    const double2 w = W[(r0 + r) * ld + col0 + c];
                    atomicMax(&eb[c], efield(w.x));
                    atomicMax(&eb[c + m], efield(w.y));
                }
            }
        }
        __syncthreads();
        // digits, transposed: Ad[s][column][row]
        for (int idx = tid; idx < kChunk * m; idx += nthr) {
            const int r = idx / m, c = idx - r * m;
            double2 y = make_double2(0.0, 0.0), w = make_double2(0.0, 0.0);
            if (r < nr) {
                y = Y[(r0 + r) * ld + col0 + c];
                if (hasW) w = W[(r0 + r) * ld + col0 + c];
            }
            uint16_t d[kS];
            split(y.x, ea[c], d);
#pragma unroll
            for (int s = 0; s < kS; ++s) Ad[((size_t)s * RP + c) * kRowStride + r] = d[s];
            split(y.y, ea[c + m], d);
#pragma unroll
            for (int s = 0; s < kS; ++s) Ad[((size_t)s * RP + c + m) * kRowStride + r] = d[s];
            if (hasW) {
                split(w.x, eb[c], d);
#pragma unroll
                for (int s = 0; s < kS; ++s) Bd[((size_t)s * RP + c) * kRowStride + r] = d[s];
                split(w.y, eb[c + m], d);
#pragma unroll
                for (int s = 0; s < kS; ++s) Bd[((size_t)s * RP + c + m) * kRowStride + r] = d[s];
            }
        }
        __syncthreads();

        for (int u = warp; u < units; u += kGramWarps) {
            const int mat = u / (MT * NG);
            const int mt = (u / NG) % MT;
            const int ng = u % NG;
            const uint16_t* Lt = Ad;                  // left operand: A^T
            const uint16_t* Rt = mat ? Bd : Ad;       // right operand: A or B
            const int* er = mat ? eb : ea;
            float acc[kS][3][4];
#pragma unroll
            for (int L = 0; L < kS; ++L)
#pragma unroll
                for (int q = 0; q < 3; ++q)
#pragma unroll
                    for (int e = 0; e < 4; ++e) acc[L][q][e] = 0.f;
#pragma unroll 1
            for (int ks = 0; ks < kChunk / 16; ++ks) {
                const int k0 = ks * 16 + tg * 2;
                uint32_t a[kS][4];
#pragma unroll
                for (int s = 0; s < kS; ++s) {
                    const uint16_t* base = Lt + ((size_t)s * RP + mt * 16 + g) * kRowStride + k0;
                    a[s][0] = ld32(base);
                    a[s][1] = ld32(base + 8 * kRowStride);
                    a[s][2] = ld32(base + 8);
                    a[s][3] = ld32(base + 8 * kRowStride + 8);
                }
#pragma unroll
                for (int t = 0; t < kS; ++t) {
                    uint32_t b[3][2];
#pragma unroll
                    for (int q = 0; q < 3; ++q) {
                        const int nt = ng * 3 + q;
                        const int n = (nt < NT ? nt : 0) * 8 + g;
                        const uint16_t* base = Rt + ((size_t)t * RP + n) * kRowStride + k0;
                        b[q][0] = ld32(base);
                        b[q][1] = ld32(base + 8);
                    }
#pragma unroll
                    for (int s = 0; s + t < kS; ++s)
#pragma unroll
                        for (int q = 0; q < 3; ++q)
                            if (ng * 3 + q < NT) mma(acc[s + t][q], a[s], b[q][0], b[q][1]);
                }
            }
            // D[mat] += level sums scaled by the chunk's column exponents
            double* Dm = D + (size_t)mat * RP * RP;
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                const int nt = ng * 3 + q;
                if (nt >= NT) continue;
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int i = mt * 16 + g + (e >> 1) * 8;
                    const int j = nt * 8 + tg * 2 + (e & 1);
                    if (i >= R2 || j >= R2) continue;
                    float c[kS];
#pragma unroll
                    for (int L = 0; L < kS; ++L) c[L] = acc[L][q][e];
                    Dm[i * RP + j] += recombine(c, ea[i], er[j]);
                }
            }
        }
    }
    __syncthreads();
    // packed upper triangles of the complex G (and S)
    const int mtri = m * (m + 1) / 2;
    const int E = nmat * mtri;
    for (int e = tid; e < E; e += nthr) {
        const int which = e / mtri;
        int k = e - which * mtri, i = 0, len = m;
        while (k >= len) { k -= len; ++i; --len; }
        const int j = i + k;
        const double* Dm = D + (size_t)which * RP * RP;
        const double re = Dm[i * RP + j] + Dm[(i + m) * RP + j + m];
        const double im = Dm[i * RP + j + m] - Dm[(i + m) * RP + j];
        partial[(size_t)blockIdx.x * E + e] = make_double2(re, im);
    }
}

// -------------------------------------------------------------- rotation
// [Re X | Im X] = [Re Y | Im Y] Qr with Qr = [[Re Q, Im Q], [-Im Q, Re Q]]
// (2m x 2mq).  Digits: per row of Y (and of W) over its 2m reals, per
// column of Qr over its 2m entries.  A CTA walks tiles of 64 rows; warp w
// owns m-tile w % 4 and n-group w / 4 (NTW n-tiles of 8 columns).  The
// tile's digits are taken before any of its rows is written, so X may
// alias Y and HX may alias W.
constexpr int kTileStride(int RK) { return RK + 8; }

struct RotSmem {
    static size_t bytes(int m, int mq) {
        const int RK = round16(2 * m), RN = round16(2 * mq);
        const size_t q = (size_t)kS * RN * kTileStride(RK) * sizeof(uint16_t);
        const size_t a = (size_t)2 * kS * kTile * kTileStride(RK) * sizeof(uint16_t);
        return q + a + (RN + 2 * kTile) * sizeof(int) + (size_t)2 * RN * sizeof(double) * 4;
    }
};

template <int NTW>
__global__ void __launch_bounds__(kRotWarps * 32, 1)
    rotate_oz_kernel(const double2* Y, const double2* W, int ld, int col0, int m, const double2* __restrict__ Q,
                     int mq, const double* __restrict__ theta, double2* X, double2* HX, long long rows,
                     double* __restrict__ res_partial) {
    extern __shared__ __align__(16) unsigned char sm[];
    const bool hasW = W != nullptr;
    const int RK = round16(2 * m), RN = round16(2 * mq), TS = kTileStride(RK);
    uint16_t* Qd = reinterpret_cast<uint16_t*>(sm);               // [kS][RN][TS]  (Qr^T digits)
    uint16_t* Yd = Qd + (size_t)kS * RN * TS;                      // [kS][kTile][TS]
    uint16_t* Wd = Yd + (size_t)kS * kTile * TS;                   // [kS][kTile][TS]
    int* fq = reinterpret_cast<int*>(Wd + (size_t)kS * kTile * TS);  // [RN] column exponents of Qr
    int* ey = fq + RN;                                             // [kTile] row exponents of Y
    int* ew = ey + kTile;                                          // [kTile] of W
    double* red = reinterpret_cast<double*>(ew + kTile);           // [4][2 RN] residual partials
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nthr = blockDim.x;
    const int g = lane >> 2, tg = lane & 3;

    // Qr digits ([t][n][k]) with per-column exponents
    for (int i = tid; i < RN; i += nthr) fq[i] = 0;
    for (int i = tid; i < kS * RN * TS; i += nthr) Qd[i] = 0;
    for (int i = tid; i < 2 * kS * kTile * TS; i += nthr) Yd[i] = 0;
    __syncthreads();
    auto qr = [&](int k, int n) -> double {
        const int i = k < m ? k : k - m, j = n < mq ? n : n - mq;
        const double2 v = Q[i * mq + j];
        if (k < m) return n < mq ? v.x : v.y;
        return n < mq ? -v.y : v.x;
    };
    for (int idx = tid; idx < 2 * m * 2 * mq; idx += nthr) {
        const int k = idx / (2 * mq), n = idx - k * (2 * mq);
        atomicMax(&fq[n], efield(qr(k, n)));
    }
    __syncthreads();
    for (int idx = tid; idx < 2 * m * 2 * mq; idx += nthr) {
        const int k = idx / (2 * mq), n = idx - k * (2 * mq);
        uint16_t d[kS];
        split(qr(k, n), fq[n], d);
#pragma unroll
        for (int t = 0; t < kS; ++t) Qd[((size_t)t * RN + n) * TS + k] = d[t];
    }

    const int mt = warp & 3, ngrp = warp >> 2;
    const int NT = RN / 8;
    double rs[NTW][2], xs[NTW][2];
#pragma unroll
    for (int q = 0; q < NTW; ++q) rs[q][0] = rs[q][1] = xs[q][0] = xs[q][1] = 0.0;

    const long long ntiles = (rows + kTile - 1) / kTile;
    const long long per = (ntiles + gridDim.x - 1) / gridDim.x;
    const long long t0 = (long long)blockIdx.x * per;
    const long long t1 = t0 + per < ntiles ? t0 + per : ntiles;
    for (long long tl = t0; tl < t1; ++tl) {
        const long long r0 = tl * kTile;
        const int nr = (int)(rows - r0 < kTile ? rows - r0 : kTile);
        __syncthreads();   // Qd ready / previous tile consumed
        // row digits: 4 threads per row, row exponent by shuffles
        {
            const int r = tid >> 2, qd = tid & 3;
            for (int pass = 0; pass < (hasW ? 2 : 1); ++pass) {
                const double2* src = pass ? W : Y;
                uint16_t* dst = pass ? Wd : Yd;
                int emax = 0;
                if (r < nr)
                    for (int c = qd; c < m; c += 4) {
                        const double2 v = src[(r0 + r) * ld + col0 + c];
                        emax = max(emax, max(efield(v.x), efield(v.y)));
                    }
                emax = max(emax, __shfl_xor_sync(0xffffffffu, emax, 1));
                emax = max(emax, __shfl_xor_sync(0xffffffffu, emax, 2));
                if (qd == 0) (pass ? ew : ey)[r] = emax;
                for (int c = qd; c < m; c += 4) {
                    const double2 v = r < nr ? src[(r0 + r) * ld + col0 + c] : make_double2(0.0, 0.0);
                    uint16_t d[kS];
                    split(v.x, emax, d);
#pragma unroll
                    for (int s = 0; s < kS; ++s) dst[((size_t)s * kTile + r) * TS + c] = d[s];
                    split(v.y, emax, d);
#pragma unroll
                    for (int s = 0; s < kS; ++s) dst[((size_t)s * kTile + r) * TS + c + m] = d[s];
                }
            }
        }
        __syncthreads();
        double xv[NTW][4];
        for (int pass = 0; pass < (hasW ? 2 : 1); ++pass) {
            const uint16_t* Ad = pass ? Wd : Yd;
            const int* er = pass ? ew : ey;
            float acc[kS][NTW][4];
#pragma unroll
            for (int L = 0; L < kS; ++L)
#pragma unroll
                for (int q = 0; q < NTW; ++q)
#pragma unroll
                    for (int e = 0; e < 4; ++e) acc[L][q][e] = 0.f;
#pragma unroll 1
            for (int ks = 0; ks < RK / 16; ++ks) {
                const int k0 = ks * 16 + tg * 2;
                uint32_t a[kS][4];
#pragma unroll
                for (int s = 0; s < kS; ++s) {
                    const uint16_t* base = Ad + ((size_t)s * kTile + mt * 16 + g) * TS + k0;
                    a[s][0] = ld32(base);
                    a[s][1] = ld32(base + 8 * TS);
                    a[s][2] = ld32(base + 8);
                    a[s][3] = ld32(base + 8 * TS + 8);
                }
#pragma unroll
                for (int t = 0; t < kS; ++t) {
                    uint32_t b[NTW][2];
#pragma unroll
                    for (int q = 0; q < NTW; ++q) {
                        const int nt = ngrp * NTW + q;
                        const int n = (nt < NT ? nt : 0) * 8 + g;
                        const uint16_t* base = Qd + ((size_t)t * RN + n) * TS + k0;
                        b[q][0] = ld32(base);
                        b[q][1] = ld32(base + 8);
                    }
#pragma unroll
                    for (int s = 0; s + t < kS; ++s)
#pragma unroll
                        for (int q = 0; q < NTW; ++q)
                            if (ngrp * NTW + q < NT) mma(acc[s + t][q], a[s], b[q][0], b[q][1]);
                }
            }
            double2* out = pass ? HX : X;
#pragma unroll
            for (int q = 0; q < NTW; ++q) {
                const int nt = ngrp * NTW + q;
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int r = mt * 16 + g + (e >> 1) * 8;
                    const int n = nt * 8 + tg * 2 + (e & 1);
                    if (nt >= NT || r >= nr || n >= 2 * mq) continue;
                    float c[kS];
#pragma unroll
                    for (int L = 0; L < kS; ++L) c[L] = acc[L][q][e];
                    const double v = recombine(c, er[r], fq[n]);
                    double* o = reinterpret_cast<double*>(out + (r0 + r) * ld + col0 + (n < mq ? n : n - mq));
                    o[n < mq ? 0 : 1] = v;
                    if (pass == 0) {
                        xv[q][e] = v;
                        xs[q][e & 1] += v * v;
                    } else if (theta) {
                        const double dv = v - theta[n < mq ? n : n - mq] * xv[q][e];
                        rs[q][e & 1] += dv * dv;
                    }
                }
            }
        }
    }
    if (!res_partial) return;
    // per-column partial sums: lanes with the same tg, then the four m-tiles
#pragma unroll
    for (int q = 0; q < NTW; ++q)
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
            for (int off = 4; off < 32; off <<= 1) {
                rs[q][h] += __shfl_xor_sync(0xffffffffu, rs[q][h], off);
                xs[q][h] += __shfl_xor_sync(0xffffffffu, xs[q][h], off);
            }
    __syncthreads();
    if (g == 0) {
#pragma unroll
        for (int q = 0; q < NTW; ++q) {
            const int nt = ngrp * NTW + q;
            if (nt >= NT) continue;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int n = nt * 8 + tg * 2 + h;
                red[(size_t)mt * 2 * RN + n] = rs[q][h];
                red[(size_t)mt * 2 * RN + RN + n] = xs[q][h];
            }
        }
    }
    __syncthreads();
    for (int j = tid; j < mq; j += nthr) {
        double a = 0.0, b = 0.0;
        for (int w = 0; w < 4; ++w) {
            a += red[(size_t)w * 2 * RN + j] + red[(size_t)w * 2 * RN + j + mq];
            b += red[(size_t)w * 2 * RN + RN + j] + red[(size_t)w * 2 * RN + RN + j + mq];
        }
        res_partial[(size_t)blockIdx.x * 2 * mq + j] = a;
        res_partial[(size_t)blockIdx.x * 2 * mq + mq + j] = b;
    }
}

static int sm_count() {
    static int n = 0;
    if (n == 0) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0)
            n = 148;
    }
    return n;
}

}  // namespace oz

bool oz_supported(int m, int mq) { return m >= 1 && mq >= 1 && m <= oz::kMaxM && mq <= oz::kMaxM; }

cudaError_t prepare_oz() {
    const int g = (int)oz::GramSmem::bytes(oz::kMaxM, true);
    const int r = (int)oz::RotSmem::bytes(oz::kMaxM, oz::kMaxM);
    cudaError_t e = cudaFuncSetAttribute(oz::gram_oz_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, g);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(oz::rotate_oz_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, r);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(oz::rotate_oz_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, r);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(oz::rotate_oz_kernel<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, r);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(oz::rotate_oz_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, r);
    return e;
}

cudaError_t launch_gram_oz(const double2* Y, const double2* W, long long rows, int ld, int col0, int m,
                           double2* partial, int nblk, double2* out, cudaStream_t st) {
    if (!oz_supported(m, m)) return cudaErrorInvalidValue;
    const long long nchunks = (rows + oz::kChunk - 1) / oz::kChunk;
    int nb = (int)std::min<long long>(std::min<long long>(nblk, oz::sm_count()), nchunks);
    if (nb < 1) nb = 1;
    const size_t smem = oz::GramSmem::bytes(m, W != nullptr);
    oz::gram_oz_kernel<<<nb, oz::kGramWarps * 32, smem, st>>>(Y, W, rows, ld, col0, m, partial);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_sum_partials_herm(partial, nb, m, W ? 2 : 1, out, st);
}

cudaError_t launch_rotate_oz(const double2* Y, const double2* W, int ld, int col0, int m, const double2* Q, int mq,
                             const double* theta, double2* X, double2* HX, long long rows, double* res_partial,
                             int nblk, double* res_out, cudaStream_t st) {
    if (!oz_supported(m, mq)) return cudaErrorInvalidValue;
    const long long ntiles = (rows + oz::kTile - 1) / oz::kTile;
    int nb = (int)std::min<long long>(std::min<long long>(nblk, oz::sm_count()), ntiles);
    if (nb < 1) nb = 1;
    const bool want_res = theta && W && res_partial && res_out;
    const size_t smem = oz::RotSmem::bytes(m, mq);
    const int NT = oz::round16(2 * mq) / 8;
    const int ntw = (NT + 1) / 2;
    double* rp = want_res ? res_partial : nullptr;
    const double* th = want_res ? theta : nullptr;
    if (ntw <= 1) oz::rotate_oz_kernel<1><<<nb, oz::kRotWarps * 32, smem, st>>>(Y, W, ld, col0, m, Q, mq, th, X, HX, rows, rp);
    else if (ntw == 2) oz::rotate_oz_kernel<2><<<nb, oz::kRotWarps * 32, smem, st>>>(Y, W, ld, col0, m, Q, mq, th, X, HX, rows, rp);
    else if (ntw == 3) oz::rotate_oz_kernel<3><<<nb, oz::kRotWarps * 32, smem, st>>>(Y, W, ld, col0, m, Q, mq, th, X, HX, rows, rp);
    else oz::rotate_oz_kernel<4><<<nb, oz::kRotWarps * 32, smem, st>>>(Y, W, ld, col0, m, Q, mq, th, X, HX, rows, rp);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || !want_res) return e;
    return launch_residual_finish(res_partial, nb, mq, res_out, st);
}

}  // namespace khp
