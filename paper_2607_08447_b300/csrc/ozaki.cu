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

#include "digits.cuh"
#include "khp_common.cuh"
#include "khp_internal.h"

namespace khp {
namespace oz {

constexpr int kMaxM = 32;       // complex columns (real width 64)
constexpr int kSub = 64;        // rows per digit tile (Gram sub-chunk, rotation tile)
constexpr int kBlkSub = 4;      // Gram: sub-chunks per exponent block (256 rows)
constexpr int kGramWarps = 12;

__host__ __device__ constexpr int round16(int v) { return (v + 15) & ~15; }
// digit-row stride in BF16 elements: an odd number of 16-B units, so the
// eight rows of an ldmatrix 8x8 load fall on distinct bank groups
__host__ __device__ constexpr int dstride(int cols) { return cols + 8; }

// Digits of v against its block's exponent field emax (|v| < 2^(emax-1022)):
// F = round(|v| 2^(49-E)) <= 2^49 = sum_s q_s 128^(6-s) with |q_s| <= 64
// for s >= 1 and 0 <= q_0 <= 128; returned as the FP32 bit patterns of
// sign(v) q_s (exact; their upper halves are the BF16 digits).  Balanced
// digits make the dropped low-level products of a value with itself (the
// Gram diagonal) average out.
__device__ __forceinline__ void split_bits(double v, int emax, uint32_t (&fb)[kS]) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    const int ex = (int)((b >> 52) & 0x7ff);
    unsigned long long F = 0;
    if (ex != 0 && emax < 2047) {
        const unsigned long long mant = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
        const int sh = emax - ex + 4;          // >= 4
        if (sh < 64) F = (mant >> sh) + ((mant >> (sh - 1)) & 1ull);
    }
    const unsigned long long G = F + kBal;
    const uint32_t neg = (uint32_t)(b >> 32) & 0x80000000u;
    // 0x4B400000 is 1.5 * 2^23: adding a small integer q to its bit pattern
    // and subtracting the float gives q exactly
    fb[0] = __float_as_uint(__int_as_float(0x4B400000 + (int)(G >> 42)) - 12582912.0f) ^ neg;
#pragma unroll
    for (int s = 1; s < kS; ++s) {
        const int u = (int)((uint32_t)(G >> (7 * (6 - s))) & 127u);
        fb[s] = __float_as_uint(__int_as_float(0x4B400000 - 64 + u) - 12582912.0f) ^ neg;
    }
}

// BF16 pair (lo at the lower address) from two FP32 bit patterns
__device__ __forceinline__ uint32_t pack_bf16(uint32_t lo, uint32_t hi) { return __byte_perm(lo, hi, 0x7632); }

__device__ __forceinline__ void mma(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
        "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// four 8x8 BF16 matrices; lane l gives the address of row l % 8 of matrix l / 8
template <bool TRANS>
__device__ __forceinline__ void ldsm4(uint32_t (&r)[4], const uint16_t* p) {
    if (TRANS)
        asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
                     : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]) : "r"(su32(p)));
    else
        asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
                     : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]) : "r"(su32(p)));
}
// two 8x8 matrices; lanes 0..15 give the row addresses (the others are ignored
// but must be valid)
template <bool TRANS>
__device__ __forceinline__ void ldsm2(uint32_t (&r)[2], const uint16_t* p) {
    if (TRANS)
        asm volatile("ldmatrix.sync.aligned.m8n8.x2.trans.shared.b16 {%0,%1}, [%2];"
                     : "=r"(r[0]), "=r"(r[1]) : "r"(su32(p)));
    else
        asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0,%1}, [%2];"
                     : "=r"(r[0]), "=r"(r[1]) : "r"(su32(p)));
}

// digits of the complex pair (a, b) of one row into a natural-layout digit
// tile D[s][row][col] (slice stride `slice`, row stride ds elements): real
// parts at columns c, c + 1, imaginary parts at m + c, m + 1 + c (m even);
// exponent fields of the four real columns
__device__ __forceinline__ void store_pair(uint16_t* D, size_t slice, int ds, int row, int c, int m, double2 a,
                                           double2 b, int ear, int ebr, int eai, int ebi) {
    uint32_t ar[kS], br[kS], ai[kS], bi[kS];
    split_bits(a.x, ear, ar);
    split_bits(b.x, ebr, br);
    split_bits(a.y, eai, ai);
    split_bits(b.y, ebi, bi);
    uint16_t* base = D + (size_t)row * ds;
#pragma unroll
    for (int s = 0; s < kS; ++s) {
        *reinterpret_cast<uint32_t*>(base + s * slice + c) = pack_bf16(ar[s], br[s]);
        *reinterpret_cast<uint32_t*>(base + s * slice + m + c) = pack_bf16(ai[s], bi[s]);
    }
}
// one complex value (m odd)
__device__ __forceinline__ void store_one(uint16_t* D, size_t slice, int ds, int row, int c, int m, double2 a,
                                          int er, int ei) {
    uint32_t ar[kS], ai[kS];
    split_bits(a.x, er, ar);
    split_bits(a.y, ei, ai);
    uint16_t* base = D + (size_t)row * ds;
#pragma unroll
    for (int s = 0; s < kS; ++s) {
        base[s * slice + c] = (uint16_t)(ar[s] >> 16);
        base[s * slice + m + c] = (uint16_t)(ai[s] >> 16);
    }
}

// ------------------------------------------------------------------ Gram
// A = [Re Y | Im Y] (rows x 2m), B = [Re W | Im W].  A CTA walks exponent
// blocks of 256 rows (64 when a warp must serve two output units): column
// exponent bounds of the block first, then four 64-row sub-chunks whose
// digits (natural layout [slice][row][column]) feed A^T A and A^T B through
// ldmatrix.trans fragments; the level sums of the whole block stay exact in
// FP32 (below 2^24) and are recombined once per block into FP64 running
// sums D in shared memory.  At the end the CTA writes the packed upper
// triangles of G_ij = D[i][j] + D[i+m][j+m] + i (D[i][j+m] - D[i+m][j])
// (and S) as its partial.  Warp unit = (matrix, 16-row m-tile, 3 n-tiles).
struct GramSmem {
    static size_t bytes(int m, bool w) {
        const int RP = round16(2 * m);
        const size_t dig = (size_t)(w ? 2 : 1) * kS * kSub * dstride(RP) * sizeof(uint16_t);
        const size_t acc = (size_t)(w ? 2 : 1) * RP * RP * sizeof(double);
        return dig + acc + 2 * RP * sizeof(int);
    }
};

__global__ void __launch_bounds__(kGramWarps * 32, 1)
    gram_oz_kernel(const double2* __restrict__ Y, const double2* __restrict__ W, long long rows, int ld, int col0,
                   int m, double2* __restrict__ partial) {
    extern __shared__ __align__(16) unsigned char sm[];
    const bool hasW = W != nullptr;
    const int nmat = hasW ? 2 : 1;
    const int R2 = 2 * m, RP = round16(R2), CS = dstride(RP);
    const size_t slice = (size_t)kSub * CS;
    uint16_t* Ad = reinterpret_cast<uint16_t*>(sm);                  // [kS][kSub][CS]
    uint16_t* Bd = Ad + kS * slice;                                  // same, W (if any)
    double* D = reinterpret_cast<double*>(Bd + (hasW ? kS * slice : 0));  // [nmat][RP][RP]
    int* ea = reinterpret_cast<int*>(D + (size_t)nmat * RP * RP);    // [RP] block column exponents of A
    int* eb = ea + RP;                                               // [RP] of B
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nthr = blockDim.x;
    const int g = lane >> 2, tg = lane & 3;

    for (int i = tid; i < nmat * RP * RP; i += nthr) D[i] = 0.0;
    // padding columns (real index >= 2m) keep zero digits for the whole run
    for (int i = tid; i < nmat * kS * (int)slice; i += nthr) Ad[i] = 0;

    const int MT = RP / 16, NT = RP / 8, NG = (NT + 2) / 3;
    const int units = nmat * MT * NG;
    const int nsub = units <= kGramWarps ? kBlkSub : 1;
    const long long BR = (long long)nsub * kSub;
    const long long nblocks = (rows + BR - 1) / BR;
    const long long per = (nblocks + gridDim.x - 1) / gridDim.x;
    const long long b0 = (long long)blockIdx.x * per;
    const long long b1 = b0 + per < nblocks ? b0 + per : nblocks;
    const int ncp = m >> 1;                 // column pairs per row
    const int items = ncp + (m & 1);        // + the single last column when m is odd

    float acc[kS][3][4];
    for (long long blk = b0; blk < b1; ++blk) {
        const long long r0 = blk * BR;
        const int nrb = (int)(rows - r0 < BR ? rows - r0 : BR);
        __syncthreads();   // previous block's digits and exponents are consumed
        for (int i = tid; i < 2 * RP; i += nthr) ea[i] = 0;
        __syncthreads();
        // column exponent bounds of the block: thread -> (column, row lane)
        {
            const int lanes = nthr / m;
            const int c = tid % m, rl = tid / m;
            if (rl < lanes) {
                int yr = 0, yi = 0, wr = 0, wi = 0;
                for (int r = rl; r < nrb; r += lanes) {
                    const double2 y = Y[(r0 + r) * ld + col0 + c];
                    yr = max(yr, efield(y.x));
                    yi = max(yi, efield(y.y));
                    if (hasW) {
                        const double2 w = W[(r0 + r) * ld + col0 + c];
                        wr = max(wr, efield(w.x));
                        wi = max(wi, efield(w.y));
                    }
                }
                atomicMax(&ea[c], yr);
                atomicMax(&ea[c + m], yi);
                if (hasW) {
                    atomicMax(&eb[c], wr);
                    atomicMax(&eb[c + m], wi);
                }
            }
        }
        if (nsub > 1) {
#pragma unroll
            for (int L = 0; L < kS; ++L)
#pragma unroll
                for (int q = 0; q < 3; ++q)
#pragma unroll
                    for (int e = 0; e < 4; ++e) acc[L][q][e] = 0.f;
        }
        for (int sub = 0; sub < nsub; ++sub) {
            const long long rs0 = r0 + (long long)sub * kSub;
            const int nr = (int)(rows - rs0 < kSub ? (rows - rs0 > 0 ? rows - rs0 : 0) : kSub);
            __syncthreads();   // exponents ready / previous sub-chunk's fragments consumed
            for (int idx = tid; idx < kSub * items; idx += nthr) {
                const int r = idx / items, k = idx - r * items;
                const bool ok = r < nr;
                if (k < ncp) {
                    const int c = 2 * k;
                    const double2* yp = Y + (rs0 + r) * ld + col0 + c;
                    const double2 y0 = ok ? yp[0] : make_double2(0.0, 0.0);
                    const double2 y1 = ok ? yp[1] : make_double2(0.0, 0.0);
                    if (m & 1) {
                        store_one(Ad, slice, CS, r, c, m, y0, ea[c], ea[c + m]);
                        store_one(Ad, slice, CS, r, c + 1, m, y1, ea[c + 1], ea[c + 1 + m]);
                    } else {
                        store_pair(Ad, slice, CS, r, c, m, y0, y1, ea[c], ea[c + 1], ea[c + m], ea[c + 1 + m]);
                    }
                    if (hasW) {
                        const double2* wp = W + (rs0 + r) * ld + col0 + c;
                        const double2 w0 = ok ? wp[0] : make_double2(0.0, 0.0);
                        const double2 w1 = ok ? wp[1] : make_double2(0.0, 0.0);
                        if (m & 1) {
                            store_one(Bd, slice, CS, r, c, m, w0, eb[c], eb[c + m]);
                            store_one(Bd, slice, CS, r, c + 1, m, w1, eb[c + 1], eb[c + 1 + m]);
                        } else {
                            store_pair(Bd, slice, CS, r, c, m, w0, w1, eb[c], eb[c + 1], eb[c + m], eb[c + 1 + m]);
                        }
                    }
                } else {
                    const int c = m - 1;
                    const double2 y = ok ? Y[(rs0 + r) * ld + col0 + c] : make_double2(0.0, 0.0);
                    store_one(Ad, slice, CS, r, c, m, y, ea[c], ea[c + m]);
                    if (hasW) {
                        const double2 w = ok ? W[(rs0 + r) * ld + col0 + c] : make_double2(0.0, 0.0);
                        store_one(Bd, slice, CS, r, c, m, w, eb[c], eb[c + m]);
                    }
                }
            }
            __syncthreads();

            for (int u = warp; u < units; u += kGramWarps) {
                const int mat = u / (MT * NG);
                const int mt = (u / NG) % MT;
                const int ng = u % NG;
                const uint16_t* Rt = mat ? Bd : Ad;
                if (nsub == 1) {
#pragma unroll
                    for (int L = 0; L < kS; ++L)
#pragma unroll
                        for (int q = 0; q < 3; ++q)
#pragma unroll
                            for (int e = 0; e < 4; ++e) acc[L][q][e] = 0.f;
                }
                const int j8 = lane >> 3, r8 = lane & 7;
                const int nt0 = ng * 3;
                const int ntA = nt0 + (j8 >> 1) < NT ? nt0 + (j8 >> 1) : 0;   // x4: tiles nt0, nt0 + 1
                const int ntB = nt0 + 2 < NT ? nt0 + 2 : 0;                   // x2: tile nt0 + 2
#pragma unroll 1
                for (int ks = 0; ks < kSub / 16; ++ks) {
                    uint32_t a[kS][4];
                    // A^T fragments from the [row][column] tile: matrix j8 = (m-block j8 & 1, k-block j8 >> 1)
                    const uint16_t* pa = Ad + (size_t)(ks * 16 + (j8 >> 1) * 8 + r8) * CS + mt * 16 + (j8 & 1) * 8;
#pragma unroll
                    for (int s = 0; s < kS; ++s) ldsm4<true>(a[s], pa + s * slice);
                    // B fragments: matrix j8 = (k-block j8 & 1, n-tile nt0 + (j8 >> 1))
                    const uint16_t* pb = Rt + (size_t)(ks * 16 + (j8 & 1) * 8 + r8) * CS + ntA * 8;
                    const uint16_t* pc = Rt + (size_t)(ks * 16 + (j8 & 1) * 8 + r8) * CS + ntB * 8;
#pragma unroll
                    for (int t = 0; t < kS; ++t) {
                        uint32_t b01[4], b2[2];
                        ldsm4<true>(b01, pb + t * slice);
                        ldsm2<true>(b2, pc + t * slice);
#pragma unroll
                        for (int s = 0; s + t < kS; ++s) {
                            if (nt0 < NT) mma(acc[s + t][0], a[s], b01[0], b01[1]);
                            if (nt0 + 1 < NT) mma(acc[s + t][1], a[s], b01[2], b01[3]);
                            if (nt0 + 2 < NT) mma(acc[s + t][2], a[s], b2[0], b2[1]);
                        }
                    }
                }
                if (nsub == 1 || sub == nsub - 1) {
                    // D[mat] += level sums scaled by the block's column exponents
                    double* Dm = D + (size_t)mat * RP * RP;
                    const int* er = mat ? eb : ea;
#pragma unroll
                    for (int q = 0; q < 3; ++q) {
                        const int nt = nt0 + q;
                        if (nt >= NT) continue;
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            const int i = mt * 16 + g + (e >> 1) * 8;
                            const int j = nt * 8 + tg * 2 + (e & 1);
                            if (i >= R2 || j >= R2) continue;
                            float c[kS];
#pragma unroll
                            for (int L = 0; L < kS; ++L) c[L] = acc[L][q][e];
                            Dm[i * RP + j] += recombine<false>(c, ea[i], er[j]);
                        }
                    }
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
// owns m-tile w % 4 and n-group w / 4 (NTW n-tiles of 8 columns), so the
// CTA has 4 ceil(NT / NTW) warps.  The
// tile's digits are taken before any of its rows is written, so X may
// alias Y and HX may alias W.  Level sums have K = 2m <= 64 terms: below
// 2^22, converted to integers without the cvt pipe.
struct RotSmem {
    static size_t bytes(int m, int mq) {
        const int RK = round16(2 * m), RN = round16(2 * mq), TS = dstride(RK);
        const size_t q = (size_t)kS * RN * TS * sizeof(uint16_t);
        const size_t a = (size_t)2 * kS * kSub * TS * sizeof(uint16_t);
        return q + a + (RN + 2 * kSub) * sizeof(int) + (size_t)4 * 2 * RN * sizeof(double);
    }
};

template <int NTW, int MAXT>
__global__ void __launch_bounds__(MAXT, 1)
    rotate_oz_kernel(const double2* Y, const double2* W, int ld, int col0, int m, const double2* __restrict__ Q,
                     int mq, const double* __restrict__ theta, double2* X, double2* HX, long long rows,
                     double* __restrict__ res_partial) {
    extern __shared__ __align__(16) unsigned char sm[];
    const bool hasW = W != nullptr;
    const int RK = round16(2 * m), RN = round16(2 * mq), TS = dstride(RK);
    const size_t slice = (size_t)kSub * TS;
    uint16_t* Qd = reinterpret_cast<uint16_t*>(sm);               // [kS][RN][TS]  (Qr^T digits)
    uint16_t* Yd = Qd + (size_t)kS * RN * TS;                      // [kS][kSub][TS]
    uint16_t* Wd = Yd + kS * slice;                                // [kS][kSub][TS]
    int* fq = reinterpret_cast<int*>(Wd + kS * slice);             // [RN] column exponents of Qr
    int* ey = fq + RN;                                             // [kSub] row exponents of Y
    int* ew = ey + kSub;                                           // [kSub] of W
    double* red = reinterpret_cast<double*>(ew + kSub);            // [4][2 RN] residual partials
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nthr = blockDim.x;
    const int g = lane >> 2, tg = lane & 3;
    const int j8 = lane >> 3, r8 = lane & 7;

    // Qr digits ([t][n][k]) with per-column exponents
    for (int i = tid; i < RN; i += nthr) fq[i] = 0;
    for (int i = tid; i < kS * RN * TS; i += nthr) Qd[i] = 0;
    for (int i = tid; i < 2 * kS * (int)slice; i += nthr) Yd[i] = 0;
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
        uint32_t d[kS];
        split_bits(qr(k, n), fq[n], d);
#pragma unroll
        for (int t = 0; t < kS; ++t) Qd[((size_t)t * RN + n) * TS + k] = (uint16_t)(d[t] >> 16);
    }

    const int mt = warp & 3, ngrp = warp >> 2;
    const int NT = RN / 8;
    double rs[NTW][2], xs[NTW][2];
#pragma unroll
    for (int q = 0; q < NTW; ++q) rs[q][0] = rs[q][1] = xs[q][0] = xs[q][1] = 0.0;
    const int ncp = m >> 1, items = ncp + (m & 1);

    const long long ntiles = (rows + kSub - 1) / kSub;
    const long long per = (ntiles + gridDim.x - 1) / gridDim.x;
    const long long t0 = (long long)blockIdx.x * per;
    const long long t1 = t0 + per < ntiles ? t0 + per : ntiles;
    for (long long tl = t0; tl < t1; ++tl) {
        const long long r0 = tl * kSub;
        const int nr = (int)(rows - r0 < kSub ? rows - r0 : kSub);
        __syncthreads();   // Qd ready / previous tile consumed
        // row digits: 4 threads per row (the first 256 threads, or every
        // thread twice for a 128-thread CTA), row exponent by shuffles
        for (int rt = tid; rt < 4 * kSub; rt += nthr) {
            const int r = rt >> 2, qd = rt & 3;
            const bool ok = r < nr;
            for (int pass = 0; pass < (hasW ? 2 : 1); ++pass) {
                const double2* src = (pass ? W : Y) + (r0 + r) * ld + col0;
                uint16_t* dst = pass ? Wd : Yd;
                int emax = 0;
                if (ok)
                    for (int c = qd; c < m; c += 4) {
                        const double2 v = src[c];
                        emax = max(emax, max(efield(v.x), efield(v.y)));
                    }
                emax = max(emax, __shfl_xor_sync(0xffffffffu, emax, 1));
                emax = max(emax, __shfl_xor_sync(0xffffffffu, emax, 2));
                if (qd == 0) (pass ? ew : ey)[r] = emax;
                for (int k = qd; k < items; k += 4) {
                    if (k < ncp) {
                        const int c = 2 * k;
                        const double2 v0 = ok ? src[c] : make_double2(0.0, 0.0);
                        const double2 v1 = ok ? src[c + 1] : make_double2(0.0, 0.0);
                        if (m & 1) {
                            store_one(dst, slice, TS, r, c, m, v0, emax, emax);
                            store_one(dst, slice, TS, r, c + 1, m, v1, emax, emax);
                        } else {
                            store_pair(dst, slice, TS, r, c, m, v0, v1, emax, emax, emax, emax);
                        }
                    } else {
                        const double2 v = ok ? src[m - 1] : make_double2(0.0, 0.0);
                        store_one(dst, slice, TS, r, m - 1, m, v, emax, emax);
                    }
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
                uint32_t a[kS][4];
                // matrix j8 = (row block j8 & 1, k-block j8 >> 1)
                const uint16_t* pa = Ad + (size_t)(mt * 16 + (j8 & 1) * 8 + r8) * TS + ks * 16 + (j8 >> 1) * 8;
#pragma unroll
                for (int s = 0; s < kS; ++s) ldsm4<false>(a[s], pa + s * slice);
#pragma unroll
                for (int t = 0; t < kS; ++t) {
                    uint32_t b[NTW][2];
#pragma unroll
                    for (int q = 0; q < NTW; q += 2) {
                        // matrix j8 = (k-block j8 & 1, n-tile q + (j8 >> 1))
                        const int ntq = ngrp * NTW + q + (q + 1 < NTW ? (j8 >> 1) : 0);
                        const int nt = ntq < NT ? ntq : 0;
                        const uint16_t* pb = Qd + ((size_t)t * RN + nt * 8 + r8) * TS + ks * 16 + (j8 & 1) * 8;
                        if (q + 1 < NTW) {
                            uint32_t r4[4];
                            ldsm4<false>(r4, pb);
                            b[q][0] = r4[0];
                            b[q][1] = r4[1];
                            b[q + 1][0] = r4[2];
                            b[q + 1][1] = r4[3];
                        } else {
                            uint32_t r2[2];
                            ldsm2<false>(r2, pb);
                            b[q][0] = r2[0];
                            b[q][1] = r2[1];
                        }
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
                    const double v = recombine<true>(c, er[r], fq[n]);
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
    if (e == cudaSuccess) e = cudaFuncSetAttribute(oz::rotate_oz_kernel<2, 384>, cudaFuncAttributeMaxDynamicSharedMemorySize, r);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(oz::rotate_oz_kernel<4, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize, r);
    return e;
}

cudaError_t launch_gram_oz(const double2* Y, const double2* W, long long rows, int ld, int col0, int m,
                           double2* partial, int nblk, double2* out, cudaStream_t st) {
    if (!oz_supported(m, m)) return cudaErrorInvalidValue;
    const long long nchunks = (rows + oz::kSub - 1) / oz::kSub;
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
    const long long ntiles = (rows + oz::kSub - 1) / oz::kSub;
    int nb = (int)std::min<long long>(std::min<long long>(nblk, oz::sm_count()), ntiles);
    if (nb < 1) nb = 1;
    const bool want_res = theta && W && res_partial && res_out;
    const size_t smem = oz::RotSmem::bytes(m, mq);
    const int NT = oz::round16(2 * mq) / 8;
    double* rp = want_res ? res_partial : nullptr;
    const double* th = want_res ? theta : nullptr;
    // two n-tiles per warp up to NT = 6 (4, 8 or 12 warps); four beyond
    if (NT <= 6) {
        const int threads = 128 * ((NT + 1) / 2);
        oz::rotate_oz_kernel<2, 384><<<nb, threads, smem, st>>>(Y, W, ld, col0, m, Q, mq, th, X, HX, rows, rp);
    } else {
        oz::rotate_oz_kernel<4, 256><<<nb, 128 * ((NT + 3) / 4), smem, st>>>(Y, W, ld, col0, m, Q, mq, th, X, HX, rows, rp);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || !want_res) return e;
    return launch_residual_finish(res_partial, nb, mq, res_out, st);
}

}  // namespace khp
