// Rayleigh-Ritz projections on the 5th-generation tensor cores (tcgen05),
// FP64 accurate: the Gram matrices G = Y^H Y, S = Y^H (H Y) and the rotation
// [X, HX] = [Y, HY] Q of every outer iteration (Sec. II B).
//
// The arithmetic is the split-digit scheme of ozaki.cu: every FP64 value of
// a block sharing an exponent bound 2^E is rounded to 49 bits below the
// bound and cut into seven balanced base-128 digits (exact in BF16); digit
// products with the same level L = s + t share one scale and are summed
// exactly in FP32; levels L <= 6 are kept and recombined in int64.  What
// changes is the machine:
//  * the CTA's threads write the digit planes into 128-byte swizzled K-major
//    shared-memory tiles (one tile per digit, M = 128 rows);
//  * one thread issues tcgen05.mma (kind::f16, BF16 x BF16 -> FP32) for every
//    digit pair, accumulating level L in TMEM columns [L N, L N + N);
//  * completion arrives on an mbarrier (tcgen05.commit); the threads read the
//    level sums with tcgen05.ld and recombine them in FP64.
// Every wait is bounded: a wait that runs out sets bit 8 of *err, the CTA
// stops issuing work, waits (bounded) for its tensor-core work in flight,
// frees its TMEM and returns.
#include <math.h>
#include <stdint.h>

#include <algorithm>

#include "digits.cuh"
#include "khp_common.cuh"
#include "khp_internal.h"
#include "tc05.cuh"

namespace khp {
namespace oztc {

using oz::kS;
using namespace tc05;

constexpr int kChunk = 64;              // rows per digit tile (the K of one Gram chunk, a rotation tile)
constexpr int kBlkChunks = 4;           // Gram: chunks per exponent block (256 rows: level sums < 2^24)
constexpr int kMaxM = 32;               // complex columns (real width 64)
constexpr uint32_t kTmemCols = 512;     // 7 levels x N <= 448 columns
constexpr size_t kMinSmem = 120 * 1024; // more than half an SM's shared memory: one CTA per SM, so
                                        // TMEM allocations never wait on another CTA
constexpr int kErrWait = 8;

__host__ __device__ constexpr int round16(int v) { return (v + 15) & ~15; }

// Balanced base-128 digits of v against its block's exponent field emax,
// from the signed integer F = sign(v) round(|v| 2^(49-E)) (E = emax - 1022):
// G = F + kBal, q_0 = G >> 42 (arithmetic), q_s = ((G >> 7(6-s)) & 127) - 64,
// so that F = sum_s q_s 128^(6-s) with |q_0| <= 128, |q_s| <= 64; returned as
// BF16 bit patterns (exact).  Zero digits for zeros, subnormals and blocks
// holding Inf/NaN (emax = 2047; the recombination returns NaN there).
__device__ __forceinline__ void split7(double v, int emax, uint32_t (&d)[kS]) {
    const long long b = __double_as_longlong(v);
    const int ex = (int)((b >> 52) & 0x7ff);
    long long F = 0;
    if (ex != 0 && emax < 2047) {
        const unsigned long long mant = ((unsigned long long)b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
        const int sh = emax - ex + 4;   // >= 4; round half up with one variable shift
        if (sh <= 64) F = (long long)(((mant >> (sh - 1)) + 1ull) >> 1);
        if (b < 0) F = -F;
    }
    const long long G = F + (long long)oz::kBal;
    // 0x4B400000 is 1.5 * 2^23: an integer q in [-2^22, 2^22) added to its
    // bit pattern gives the float 1.5 * 2^23 + q exactly
    d[0] = __float_as_uint(__int_as_float(0x4B400000 + (int)(G >> 42)) - 12582912.0f) >> 16;
#pragma unroll
    for (int s = 1; s < kS; ++s) {
        const uint32_t u = (uint32_t)(G >> (7 * (6 - s))) & 127u;
        d[s] = __float_as_uint(__int_as_float((int)(0x4B400000u | u)) - 12582976.0f) >> 16;
    }
}

__device__ __forceinline__ uint32_t pack2(uint32_t lo, uint32_t hi) { return lo | (hi << 16); }

// ------------------------------------------------------------------ Gram
// A level tile holds the digits of one level for the real columns of Y
// (rows 0 .. 2m-1, padded to RP) and of W (rows RP .. RP + 2m - 1), K = the
// 64 grid rows of a chunk.  The product of level-s tile rows [0, 128) with
// level-t tile rows [0, RP) (the Y columns) gives, for one digit pair,
//   D[i][j] = sum_k A_s[i][k] Y_t[j][k]:  Y^T Y for i < RP, W^T Y for i >= RP.
// Rows past RA of the M = 128 operand read the next tile (ignored rows), so a
// buffer is 7 tiles plus the 128 - RA rows the last read runs past.
//
// Roles: warp 0 issues the products (lane 0); warps 1.. ("producers") take
// the block exponent bounds and write the digit tiles one chunk ahead of the
// products, into two alternating buffers when shared memory holds two (one
// otherwise).  Exponent blocks of 256 rows: while warp 0 issues a block's
// last chunk, the producers take the next block's column exponent bounds
// (its rows were prefetched into L2 when the block before it started); then
// every warp reads level sums from TMEM (warp w: lanes 32 (w % 4) + lane,
// column quarter w / 4) and adds their FP64 recombination to running sums in
// shared memory.
constexpr int kGThreads = 512;
constexpr int kProducers = kGThreads - 32;
constexpr int kItemsP = (2 * 4 * (kMaxM / 8) * 32 + kProducers - 1) / kProducers;   // split items per producer (3)

// G = F + kBal for the balanced digits of split7 (64-bit, two registers)
__device__ __forceinline__ long long balanced(double v, int emax) {
    const long long b = __double_as_longlong(v);
    const int ex = (int)((b >> 52) & 0x7ff);
    long long F = 0;
    if (ex != 0 && emax < 2047) {
        const unsigned long long mant = ((unsigned long long)b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
        const int sh = emax - ex + 4;   // round half up with one variable shift
        if (sh <= 64) F = (long long)(((mant >> (sh - 1)) + 1ull) >> 1);
        if (b < 0) F = -F;
    }
    return F + (long long)oz::kBal;
}
// BF16 bit pattern of digit s of G (as split7)
template <int S>
__device__ __forceinline__ uint32_t digit(long long G) {
    if (S == 0) return __float_as_uint(__int_as_float(0x4B400000 + (int)(G >> 42)) - 12582912.0f) >> 16;
    const uint32_t u = (uint32_t)(G >> (7 * (6 - S))) & 127u;
    return __float_as_uint(__int_as_float((int)(0x4B400000u | u)) - 12582976.0f) >> 16;
}

struct GramGeo {
    int RP, RA, nbuf;
    size_t tile, buf, acc;
    __host__ __device__ GramGeo(int m, bool w)
        : RP(round16(2 * m)), RA((w ? 2 : 1) * round16(2 * m)), nbuf(2), tile((size_t)RA * 128),
          buf((size_t)(6 * RA + 128) * 128), acc((size_t)(w ? 2 : 1) * round16(2 * m) * (round16(2 * m) + 1) * 8) {
        if (bytes(2) > kSmemMax) nbuf = 1;
    }
    __host__ __device__ size_t bytes(int nb) const { return 1024 + nb * buf + acc + 2 * 128 * sizeof(int) + 64; }
    __host__ __device__ size_t smem() const { return bytes(nbuf); }
    static constexpr size_t kSmemMax = 227 * 1024;
};

__device__ __forceinline__ void ld4(uint32_t taddr, float (&v)[4]) {
    uint32_t r[4];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(taddr));
#pragma unroll
    for (int i = 0; i < 4; ++i) v[i] = __uint_as_float(r[i]);
}

__global__ void __launch_bounds__(kGThreads, 1)
    gram_tc_kernel(const double2* __restrict__ Y, const double2* __restrict__ W, long long rows, int ld, int col0,
                   int m, double2* __restrict__ partial, int* err) {
    extern __shared__ __align__(1024) unsigned char sm_raw[];
    const uint32_t s_raw = saddr(sm_raw);
    unsigned char* sm = sm_raw + (((s_raw + 1023u) & ~1023u) - s_raw);
    const bool hasW = W != nullptr;
    const int nmat = hasW ? 2 : 1;
    const GramGeo geo(m, hasW);
    const int RP = geo.RP, nbuf = geo.nbuf;
    const int RD = RP + 1;   // running-sum row stride (odd: the lanes of a warp, one row each, hit distinct banks)
    unsigned char* dig = sm;                                          // [nbuf][buf]
    double* D = reinterpret_cast<double*>(dig + nbuf * geo.buf);     // [nmat][RP][RD] FP64 running sums
    int* ea = reinterpret_cast<int*>(reinterpret_cast<unsigned char*>(D) + geo.acc);   // [2][128] block exponents
    uint64_t* bars = reinterpret_cast<uint64_t*>(ea + 2 * 128);       // [2] one per digit buffer
    uint32_t* tslot = reinterpret_cast<uint32_t*>(bars + 2);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int ptid = tid - 32;                                        // producer index (< 0 in warp 0)

    // padding rows and the slack stay zero for the whole run
    for (size_t i = tid; i < nbuf * geo.buf / 16; i += kGThreads)
        reinterpret_cast<uint4*>(dig)[i] = make_uint4(0u, 0u, 0u, 0u);
    for (size_t i = tid; i < geo.acc / 8; i += kGThreads) D[i] = 0.0;
    for (int i = tid; i < 2 * 128; i += kGThreads) ea[i] = 0;
    if (warp == 0) tmem_alloc(tslot, kTmemCols);
    if (tid == 0) {
        mbar_init(saddr(&bars[0]), 1);
        mbar_init(saddr(&bars[1]), 1);
    }
    fence_proxy_async();
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tslot;

    const long long BR = (long long)kBlkChunks * kChunk;
    const long long nblocks = (rows + BR - 1) / BR;
    const long long per = (nblocks + gridDim.x - 1) / gridDim.x;
    const long long b0 = (long long)blockIdx.x * per;
    const long long b1 = b0 + per < nblocks ? b0 + per : nblocks;

    // the rows of a block into L2 (producers)
    auto prefetch_block = [&](long long blk) {
        if (ptid < 0 || blk >= b1) return;
        const long long r0 = blk * BR;
        const int nrb = (int)(rows - r0 < BR ? rows - r0 : BR);
        for (int i = ptid; i < nmat * nrb; i += kProducers) {
            const int mat = i / nrb, r = i - mat * nrb;
            prefetch_l2((mat ? W : Y) + (r0 + r) * ld + col0, (uint32_t)(m * 16));
        }
    };
    // column exponent bounds of a block into e (producers; e zeroed before)
    const int nexp = nmat * m;
    const int elanes = kProducers / nexp;
    auto exponents = [&](long long blk, int* e) {
        const long long r0 = blk * BR;
        const int nrb = (int)(rows - r0 < BR ? rows - r0 : BR);
        const int task = ptid % nexp, rl = ptid / nexp;
        if (ptid < 0 || rl >= elanes) return;
        const int mat = task / m, cc = task - mat * m;
        const double2* src = (mat ? W : Y) + col0 + cc;
        int er = 0, ei = 0;
        for (int rb = rl; rb < nrb; rb += 8 * elanes) {
            double2 v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int r = rb + u * elanes;
                v[u] = r < nrb ? src[(r0 + r) * ld] : make_double2(0.0, 0.0);
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                er = max(er, oz::efield(v[u].x));
                ei = max(ei, oz::efield(v[u].y));
            }
        }
        atomicMax(&e[mat * RP + cc], er);
        atomicMax(&e[mat * RP + m + cc], ei);
    };
    // products of one chunk's digit buffer (warp 0, lane 0)
    const uint32_t idesc = idesc_bf16(128, RP);
    const uint64_t tstep = (uint64_t)(geo.tile >> 4);
    // chunk k's products commit to bars[k % nbuf]: completion k / nbuf of that barrier
    auto bar_of = [&](long long k) { return saddr(&bars[k % nbuf]); };
    auto par_of = [&](long long k) { return (uint32_t)((k / nbuf) & 1); };
    auto issue = [&](int bsel, bool first) {
        fence_after();
        const uint64_t d0 = desc_sw128(saddr(dig + (size_t)bsel * geo.buf));
#pragma unroll
        for (int ks = 0; ks < kChunk / 16; ++ks)
#pragma unroll
            for (int s = 0; s < kS; ++s) {
                const uint64_t ad = d0 + (uint64_t)s * tstep + 2u * ks;
#pragma unroll
                for (int t = 0; s + t < kS; ++t)
                    mma_bf16(tmem + (uint32_t)((s + t) * RP), ad, d0 + (uint64_t)t * tstep + 2u * ks, idesc,
                             !(first && ks == 0 && s == 0));
            }
        commit(saddr(&bars[bsel]));
    };

    // recombination: A row i (Y column i, or W column i - RP), column quarter w / 4 of RP
    const int i_row = 32 * (warp & 3) + lane;
    const int nq = RP / 4, jb = (warp >> 2) * nq;
    const bool vrow = i_row < 2 * m || (hasW && i_row >= RP && i_row < RP + 2 * m);
    const uint32_t tl = tmem + ((uint32_t)(32 * (warp & 3)) << 16);
    double* Drow = D + (size_t)(i_row < RP ? 0 : 1) * RP * RD + (size_t)(i_row < RP ? i_row : i_row - RP) * RD;

    // split items (matrix, 4-row group k4, complex column cc): a warp's 32
    // lanes take 8 consecutive columns (lane & 7) of 4 consecutive groups
    // (lane >> 3), so that its 8-byte digit stores spread over the banks;
    // item groups of 32: (matrix, k4 / 4, column octet)
    const int ncg = (m + 7) / 8;
    const int nitems = nmat * 4 * ncg * 32;
    auto item = [&](int it, int& mat, int& k4, int& cc) {
        const int l = it & 31, grp = it >> 5;
        const int cg = grp % ncg, rest = grp / ncg;
        const int k4hi = rest & 3;
        mat = rest >> 2;
        k4 = 4 * k4hi + (l >> 3);
        cc = 8 * cg + (l & 7);
    };
    long long c = 0;                    // chunks split so far
    long long ncommit = 0;              // chunks whose products were issued
    bool failed = false;

    if (b0 < b1) {
        prefetch_block(b0);
        exponents(b0, ea);
    }
    __syncthreads();
    for (long long blk = b0; blk < b1 && !failed; ++blk) {
        int* eac = ea + ((blk - b0) & 1) * 128;
        int* ean = ea + (((blk - b0) & 1) ^ 1) * 128;
        const long long r0 = blk * BR;
        const int nrb = (int)(rows - r0 < BR ? rows - r0 : BR);
        const int nsub = (nrb + kChunk - 1) / kChunk;
        prefetch_block(blk + 1);
        for (int sub = 0; sub < nsub; ++sub, ++c) {
            bool ok = true;
            if (warp == 0) {
                // two buffers: the previous chunk of this block, while this one is split
                if (nbuf == 2 && lane == 0 && sub > 0) issue((int)((c - 1) % nbuf), sub == 1);
            } else {
                const int bsel = (int)(c % nbuf);
                // the tensor cores are done with chunk c - nbuf (same buffer); with one
                // buffer the previous chunk's products were issued before the last barrier
                if (c >= nbuf) ok = mbar_wait(bar_of(c - nbuf), par_of(c - nbuf));
                unsigned char* bufp = dig + (size_t)bsel * geo.buf;
                const long long rs0 = r0 + (long long)sub * kChunk;
                const int nr = (int)(rows - rs0 < kChunk ? rows - rs0 : kChunk);
                double2 va[kItemsP][4];
#pragma unroll
                for (int u = 0; u < kItemsP; ++u) {
                    const int it = ptid + u * kProducers;
                    int mat, k4, cc;
                    item(it, mat, k4, cc);
                    if (it < nitems && cc < m) {
                        const double2* src = (mat ? W : Y) + (rs0 + 4 * k4) * ld + col0 + cc;
#pragma unroll
                        for (int q = 0; q < 4; ++q)
                            va[u][q] = 4 * k4 + q < nr ? src[(long long)q * ld] : make_double2(0.0, 0.0);
                    }
                }
#pragma unroll
                for (int u = 0; u < kItemsP; ++u) {
                    const int it = ptid + u * kProducers;
                    if (it >= nitems) break;
                    int mat, k4, cc;
                    item(it, mat, k4, cc);
                    if (cc >= m) continue;
                    const int rre = mat * RP + cc, rim = mat * RP + m + cc;
                    const int er = eac[rre], ei = eac[rim];
                    long long gr[4], gi[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        gr[q] = balanced(va[u][q].x, er);
                        gi[q] = balanced(va[u][q].y, ei);
                    }
                    unsigned char* pre = bufp + sw128_chunk(rre, k4 >> 1) + 8u * (k4 & 1);
                    unsigned char* pim = bufp + sw128_chunk(rim, k4 >> 1) + 8u * (k4 & 1);
#define KHP_STORE_LEVEL(S)                                                                                  \
    *reinterpret_cast<uint2*>(pre + (size_t)(S) * geo.tile) =                                               \
        make_uint2(pack2(digit<S>(gr[0]), digit<S>(gr[1])), pack2(digit<S>(gr[2]), digit<S>(gr[3])));       \
    *reinterpret_cast<uint2*>(pim + (size_t)(S) * geo.tile) =                                               \
        make_uint2(pack2(digit<S>(gi[0]), digit<S>(gi[1])), pack2(digit<S>(gi[2]), digit<S>(gi[3])));
                    KHP_STORE_LEVEL(0)
                    KHP_STORE_LEVEL(1)
                    KHP_STORE_LEVEL(2)
                    KHP_STORE_LEVEL(3)
                    KHP_STORE_LEVEL(4)
                    KHP_STORE_LEVEL(5)
                    KHP_STORE_LEVEL(6)
#undef KHP_STORE_LEVEL
                }
                fence_proxy_async();
            }
            if (nbuf == 2 && sub > 0) ++ncommit;
            if (__syncthreads_or(!ok)) { failed = true; break; }
            if (nbuf == 1 && sub + 1 < nsub) {
                // one buffer: this chunk's products run before the next chunk is split
                if (warp == 0 && lane == 0) issue(0, sub == 0);
                ++ncommit;
                const bool ok1 = mbar_wait(bar_of(c), par_of(c));
                if (__syncthreads_or(!ok1)) { failed = true; break; }
            }
        }
        if (failed) break;
        // warp 0 issues the block's last chunk while the producers take the
        // next block's exponent bounds
        if (warp == 0) {
            if (lane == 0) issue((int)((c - 1) % nbuf), nsub == 1);
        } else if (blk + 1 < b1) {
            for (int i = ptid; i < 128; i += kProducers) ean[i] = 0;
            asm volatile("bar.sync 1, %0;" ::"r"(kProducers) : "memory");
            exponents(blk + 1, ean);
        }
        ++ncommit;
        {
            const bool ok = mbar_wait(bar_of(c - 1), par_of(c - 1));
            if (__syncthreads_or(!ok)) { failed = true; break; }
        }
        fence_after();
        const int erow = eac[i_row];
        for (int p = 0; p < nq; p += 4) {
            float cv[kS][4];
#pragma unroll
            for (int L = 0; L < kS; ++L) ld4(tl + (uint32_t)(L * RP + jb + p), cv[L]);
            wait_ld();
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int j = jb + p + q;
                if (vrow && j < 2 * m) {
                    float cl[kS];
#pragma unroll
                    for (int L = 0; L < kS; ++L) cl[L] = cv[L][q];
                    Drow[j] += oz::recombine<false>(cl, erow, eac[j]);
                }
            }
        }
        fence_before();
        __syncthreads();   // TMEM read and eac consumed before the next block's products
    }

    if (failed) {
        if (tid == 0) atomicOr(err, kErrWait);
        // bounded wait for the products in flight before the TMEM is freed
        if (ncommit > 0) mbar_wait(bar_of(ncommit - 1), par_of(ncommit - 1));
    }
    __syncthreads();
    // packed upper triangles of the complex G (and S) from the running sums:
    // D0[i][j] = Y_i . Y_j and D1[a][j] = W_a . Y_j (real columns)
    const int mtri = m * (m + 1) / 2;
    const int E = nmat * mtri;
    for (int e = tid; e < E; e += kGThreads) {
        const int which = e / mtri;
        int k = e - which * mtri, i = 0, len = m;
        while (k >= len) { k -= len; ++i; --len; }
        const int j = i + k;
        double re, im;
        if (which == 0) {
            const double* Dm = D;
            re = Dm[i * RD + j] + Dm[(i + m) * RD + j + m];
            im = Dm[i * RD + j + m] - Dm[(i + m) * RD + j];
        } else {
            // S_ij = sum_k conj(Y_ki) W_kj:  with T[a][b] = W_a . Y_b,
            // Re = T[j][i] + T[j+m][i+m], Im = T[j+m][i] - T[j][i+m]
            const double* T = D + (size_t)RP * RD;
            re = T[j * RD + i] + T[(j + m) * RD + i + m];
            im = T[(j + m) * RD + i] - T[j * RD + i + m];
        }
        partial[(size_t)blockIdx.x * E + e] = make_double2(re, im);
    }
    fence_before();
    __syncthreads();
    if (warp == 0) {
        fence_after();
        tmem_dealloc(tmem, kTmemCols);
    }
}

// -------------------------------------------------------------- rotation
// [X, HX] = [Y, W] Q in the interleaved real form: K index 2c + q (q = 0
// real, 1 imaginary part of input column c), output column n = 2j + p (p = 0
// real, 1 imaginary part of X_j), with
//   Qr^T[2j][2c] = Re Q_cj, Qr^T[2j][2c+1] = -Im Q_cj,
//   Qr^T[2j+1][2c] = Im Q_cj, Qr^T[2j+1][2c+1] = Re Q_cj,
// so that a row's reals are in memory order.  A tile of 64 grid rows: the
// A operand holds the Y rows (M rows 0..63) and the W rows (64..127) with a
// row exponent each, B the digits of Qr^T (RN rows, a column exponent each,
// taken once per CTA); the Qr^T planes are contiguous, so one product takes
// up to 256 / RN planes.  The level sums go through FP64 recombination into
// a staging area, from which the rows are written out coalesced along with
// the residual partial sums.  When shared memory holds a separate staging
// area, tile i's rows are written out while the tensor cores multiply tile
// i + 1; otherwise the staging area is the A tiles' memory.
constexpr int kRThreads = 512;

struct RotGeo {
    int RK, RN, SS;
    bool sep;
    size_t atile, qtile, stage;
    __host__ __device__ RotGeo(int m, int mq)
        : RK(round16(2 * m)), RN(round16(2 * mq)), SS(round16(2 * mq) + 1), sep(true), atile((size_t)128 * 128),
          qtile((size_t)round16(2 * mq) * 128), stage((size_t)2 * 64 * (round16(2 * mq) + 1) * 8) {
        if (bytes(true) > GramGeo::kSmemMax) sep = false;
    }
    __host__ __device__ size_t bytes(bool s) const {
        return 1024 + kS * atile + kS * qtile + (s ? stage : 0) + (64 + 128) * sizeof(int) +
               (size_t)kRThreads * 2 * sizeof(float) + 64;
    }
    __host__ __device__ size_t smem() const { return bytes(sep); }
};

// float close to |v| (top 20 mantissa bits; 0 below 2^-126): integer
// operations only, for the residual norms, which need a few digits
__device__ __forceinline__ float approx_abs_f(double v) {
    const unsigned int hi = (unsigned int)((unsigned long long)__double_as_longlong(v) >> 32) & 0x7fffffffu;
    const int e = (int)(hi >> 20) - 896;
    if (e <= 0) return 0.0f;
    if (e >= 255) return __int_as_float(0x7f800000);
    return __uint_as_float(((unsigned int)e << 23) | ((hi & 0xFFFFFu) << 3));
}

// the recombination of oz::recombine<true> as one int64 when it fits (the
// usual case), without the FP64 addition of the two parts
__device__ __forceinline__ double recombine_small(const float (&c)[kS], int ea, int eb) {
    if (ea == 2047 || eb == 2047) return __longlong_as_double(0x7ff8000000000000ll);
    long long hi = 0, lo = 0;
#pragma unroll
    for (int L = 0; L < 4; ++L) hi = hi * 128 + oz::f2ll<true>(c[L]);
#pragma unroll
    for (int L = 4; L < kS; ++L) lo = lo * 128 + oz::f2ll<true>(c[L]);
    const int E = (ea - 1022) + (eb - 1022) - 14;
    if (hi < (1ll << 41) && hi > -(1ll << 41)) return oz::i2d_scaled(hi * (1ll << 21) + lo, E - 42);
    return oz::i2d_scaled(hi, E - 21) + oz::i2d_scaled(lo, E - 42);
}

__global__ void __launch_bounds__(kRThreads, 1)
    rotate_tc_kernel(const double2* Y, const double2* W, int ld, int col0, int m, const double2* __restrict__ Q,
                     int mq, const double* __restrict__ theta, double2* X, double2* HX, long long rows,
                     double* __restrict__ res_partial, int* err) {
    extern __shared__ __align__(1024) unsigned char sm_raw[];
    const uint32_t s_raw = saddr(sm_raw);
    unsigned char* sm = sm_raw + (((s_raw + 1023u) & ~1023u) - s_raw);
    const bool hasW = W != nullptr;
    const RotGeo geo(m, mq);
    const int RK = geo.RK, RN = geo.RN, SS = geo.SS;
    const bool sep = geo.sep;
    unsigned char* adig = sm;                                         // [kS][128 rows][128 B]
    unsigned char* qdig = adig + kS * geo.atile;                      // [kS][RN rows][128 B]
    double* stage = reinterpret_cast<double*>(sep ? qdig + kS * geo.qtile : adig);   // [2][64][SS]
    int* fq = reinterpret_cast<int*>(qdig + kS * geo.qtile + (sep ? geo.stage : 0));   // [64] Qr^T column exponents
    int* ey = fq + 64;                                                // [128] row exponents (Y, then W)
    float* red = reinterpret_cast<float*>(ey + 128);                  // [kRThreads][2] residual partials
    uint64_t* bar = reinterpret_cast<uint64_t*>(red + 2 * kRThreads);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 1);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    for (size_t i = tid; i < (kS * geo.atile + kS * geo.qtile) / 16; i += kRThreads)
        reinterpret_cast<uint4*>(adig)[i] = make_uint4(0u, 0u, 0u, 0u);
    for (int i = tid; i < 64; i += kRThreads) fq[i] = 0;
    if (warp == 0) tmem_alloc(tslot, kTmemCols);
    if (tid == 0) mbar_init(saddr(bar), 1);
    __syncthreads();
    // Qr^T digits, one exponent per output column
    auto qr = [&](int n, int k) -> double {
        const int j = n >> 1, p = n & 1, cidx = k >> 1, q = k & 1;
        const double2 v = Q[cidx * mq + j];
        if (p == 0) return q == 0 ? v.x : -v.y;
        return q == 0 ? v.y : v.x;
    };
    for (int idx = tid; idx < 2 * mq * 2 * m; idx += kRThreads) {
        const int n = idx / (2 * m), k = idx - n * (2 * m);
        atomicMax(&fq[n], oz::efield(qr(n, k)));
    }
    __syncthreads();
    for (int idx = tid; idx < 2 * mq * (RK / 8); idx += kRThreads) {
        const int n = idx / (RK / 8), k8 = idx - n * (RK / 8);
        uint32_t d[8][kS];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const int k = 8 * k8 + e;
            split7(k < 2 * m ? qr(n, k) : 0.0, fq[n], d[e]);
        }
#pragma unroll
        for (int t = 0; t < kS; ++t)
            *reinterpret_cast<uint4*>(qdig + (size_t)t * geo.qtile + sw128_chunk(n, k8)) =
                make_uint4(pack2(d[0][t], d[1][t]), pack2(d[2][t], d[3][t]), pack2(d[4][t], d[5][t]),
                           pack2(d[6][t], d[7][t]));
    }
    fence_proxy_async();
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tslot;

    // output items: thread -> fixed column oj, rows orl, orl + tpc, ...
    const int tpc = kRThreads / mq;
    const int oj = tid % mq, orl = tid / mq;
    const double th = (theta && orl < tpc) ? theta[oj] : 0.0;
    float rsum = 0.f, xsum = 0.f;
    auto output = [&](long long r0, int nr) {
        if (orl >= tpc) return;
        for (int r = orl; r < nr; r += tpc) {
            const double2 xv = make_double2(stage[(size_t)r * SS + 2 * oj], stage[(size_t)r * SS + 2 * oj + 1]);
            X[(r0 + r) * ld + col0 + oj] = xv;
            if (hasW) {
                const size_t o = ((size_t)64 + r) * SS + 2 * oj;
                const double2 hv = make_double2(stage[o], stage[o + 1]);
                HX[(r0 + r) * ld + col0 + oj] = hv;
                if (theta) {
                    // the difference in FP64, its square and |x|^2 in FP32
                    const float dr = approx_abs_f(fma(-th, xv.x, hv.x)), di = approx_abs_f(fma(-th, xv.y, hv.y));
                    const float ax = approx_abs_f(xv.x), ay = approx_abs_f(xv.y);
                    rsum = fmaf(dr, dr, fmaf(di, di, rsum));
                    xsum = fmaf(ax, ax, fmaf(ay, ay, xsum));
                }
            }
        }
    };

    const int i_row = 32 * (warp & 3) + lane;    // TMEM lane = A row (Y rows, then W rows)
    const int nq = RN / 4, nb0 = (warp >> 2) * nq;
    const uint32_t tl = tmem + ((uint32_t)(32 * (warp & 3)) << 16);
    // split mapping: thread -> (matrix, row, quad lane)
    const int smat = tid >> 8, srow = (tid & 255) >> 2, sqd = tid & 3;

    const long long ntiles = (rows + kChunk - 1) / kChunk;
    const long long per = (ntiles + gridDim.x - 1) / gridDim.x;
    const long long t0 = (long long)blockIdx.x * per;
    const long long t1 = t0 + per < ntiles ? t0 + per : ntiles;
    long long issued = 0;
    long long prev_r0 = 0;
    int prev_nr = 0;
    bool failed = false;
    for (long long tl_i = t0; tl_i < t1; ++tl_i) {
        const long long r0 = tl_i * kChunk;
        const int nr = (int)(rows - r0 < kChunk ? rows - r0 : kChunk);
        if (tl_i + 1 < t1 && tid < 2 * kChunk) {
            // the next tile's rows into L2
            const int mat = tid / kChunk, r = tid - mat * kChunk;
            const long long rn = r0 + kChunk + r;
            if (rn < rows && (mat == 0 || hasW)) prefetch_l2((mat ? W : Y) + rn * ld + col0, (uint32_t)(m * 16));
        }
        __syncthreads();   // the A tiles (and a staging area in them) are free
        // row digits: the quad (matrix, row) splits the row's 16-byte chunks
        // qd and qd + 4 (4 complex values each), every load issued first
        if (smat == 0 || hasW) {
            const double2* src = (smat ? W : Y) + (r0 + srow) * ld + col0;
            const bool ok = srow < nr;
            double2 v[2][4];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int k8 = sqd + 4 * h;
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int cidx = 4 * k8 + e;
                    v[h][e] = (ok && k8 < RK / 8 && cidx < m) ? src[cidx] : make_double2(0.0, 0.0);
                }
            }
            int emax = 0;
#pragma unroll
            for (int h = 0; h < 2; ++h)
#pragma unroll
                for (int e = 0; e < 4; ++e) emax = max(emax, max(oz::efield(v[h][e].x), oz::efield(v[h][e].y)));
            emax = max(emax, __shfl_xor_sync(0xffffffffu, emax, 1));
            emax = max(emax, __shfl_xor_sync(0xffffffffu, emax, 2));
            if (sqd == 0) ey[smat * 64 + srow] = emax;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int k8 = sqd + 4 * h;
                if (k8 >= RK / 8) continue;
                long long g[8];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    g[2 * e] = balanced(v[h][e].x, emax);
                    g[2 * e + 1] = balanced(v[h][e].y, emax);
                }
                unsigned char* dst = adig + sw128_chunk(smat * 64 + srow, k8);
#define KHP_STORE_LEVEL(S)                                                                                   \
    *reinterpret_cast<uint4*>(dst + (size_t)(S) * geo.atile) =                                               \
        make_uint4(pack2(digit<S>(g[0]), digit<S>(g[1])), pack2(digit<S>(g[2]), digit<S>(g[3])),             \
                   pack2(digit<S>(g[4]), digit<S>(g[5])), pack2(digit<S>(g[6]), digit<S>(g[7])));
                KHP_STORE_LEVEL(0)
                KHP_STORE_LEVEL(1)
                KHP_STORE_LEVEL(2)
                KHP_STORE_LEVEL(3)
                KHP_STORE_LEVEL(4)
                KHP_STORE_LEVEL(5)
                KHP_STORE_LEVEL(6)
#undef KHP_STORE_LEVEL
            }
        }
        fence_proxy_async();
        __syncthreads();
        if (tid == 0) {
            // the Qr^T planes are contiguous: one product takes up to kp
            // planes t0 .. t0 + kp - 1 (N <= 256), landing on the level
            // columns (s + t) RN
            fence_after();
            const uint64_t da = desc_sw128(saddr(adig)), dq = desc_sw128(saddr(qdig));
            const uint64_t astep = (uint64_t)(geo.atile >> 4), qstep = (uint64_t)(geo.qtile >> 4);
            const int kp = 256 / RN;
#pragma unroll 1
            for (int ks = 0; ks < RK / 16; ++ks) {
#pragma unroll 1
                for (int s = 0; s < kS; ++s) {
                    const uint64_t ad = da + (uint64_t)s * astep + 2u * ks;
#pragma unroll 1
                    for (int tp = 0; tp < kS - s; tp += kp) {
                        const int np = kS - s - tp < kp ? kS - s - tp : kp;
                        mma_bf16(tmem + (uint32_t)((s + tp) * RN), ad, dq + (uint64_t)tp * qstep + 2u * ks,
                                 idesc_bf16(128, np * RN), !(ks == 0 && s == 0));
                    }
                }
            }
            commit(saddr(bar));
        }
        ++issued;
        // the previous tile's rows go out while the tensor cores work
        if (sep && tl_i > t0) output(prev_r0, prev_nr);
        {
            const bool ok = mbar_wait(saddr(bar), (uint32_t)((issued - 1) & 1));
            if (__syncthreads_or(!ok)) { failed = true; break; }
        }
        fence_after();
        // level sums -> FP64 in the staging area
        {
            const int erow = ey[i_row];
            const int mat = i_row >> 6, r = i_row & 63;
            for (int p = 0; p < nq; p += 4) {
                float cv[kS][4];
#pragma unroll
                for (int L = 0; L < kS; ++L) ld4(tl + (uint32_t)(L * RN + nb0 + p), cv[L]);
                wait_ld();
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int n = nb0 + p + q;
                    float cl[kS];
#pragma unroll
                    for (int L = 0; L < kS; ++L) cl[L] = cv[L][q];
                    stage[((size_t)mat * 64 + r) * SS + n] = recombine_small(cl, erow, fq[n]);
                }
            }
        }
        fence_before();
        __syncthreads();
        if (!sep) output(r0, nr);
        prev_r0 = r0;
        prev_nr = nr;
    }
    if (failed) {
        if (tid == 0) atomicOr(err, kErrWait);
        // bounded wait for the products in flight before the TMEM is freed
        mbar_wait(saddr(bar), (uint32_t)((issued - 1) & 1));
    } else if (sep && t1 > t0) {
        output(prev_r0, prev_nr);
    }
    __syncthreads();
    if (res_partial) {
        red[2 * tid] = rsum;
        red[2 * tid + 1] = xsum;
        __syncthreads();
        for (int j = tid; j < mq; j += kRThreads) {
            double a = 0.0, b = 0.0;
            for (int q = 0; q < tpc; ++q) {
                a += (double)red[2 * (q * mq + j)];
                b += (double)red[2 * (q * mq + j) + 1];
            }
            res_partial[(size_t)blockIdx.x * 2 * mq + j] = a;
            res_partial[(size_t)blockIdx.x * 2 * mq + mq + j] = b;
        }
    }
    fence_before();
    __syncthreads();
    if (warp == 0) {
        fence_after();
        tmem_dealloc(tmem, kTmemCols);
    }
}

static int sm_count() {
    static int n = 0;
    if (n == 0) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0)
            n = 148;
    }
    return n;
}

}  // namespace oztc

bool tc_supported(int m, int mq) { return m >= 1 && mq >= 1 && m <= oztc::kMaxM && mq <= oztc::kMaxM; }

cudaError_t prepare_tc() {
    int g = 0;
    for (int m = 1; m <= oztc::kMaxM; ++m)
        for (int w = 0; w < 2; ++w) g = std::max(g, (int)oztc::GramGeo(m, w != 0).smem());
    int r = (int)oztc::kMinSmem;
    for (int m = 1; m <= oztc::kMaxM; ++m) r = std::max(r, (int)oztc::RotGeo(m, m).smem());
    cudaError_t e = cudaFuncSetAttribute(oztc::gram_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, g);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(oztc::rotate_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, r);
    return e;
}

cudaError_t launch_gram_tc(const double2* Y, const double2* W, long long rows, int ld, int col0, int m,
                           double2* partial, int nblk, double2* out, int* err, cudaStream_t st) {
    if (!tc_supported(m, m) || !err) return cudaErrorInvalidValue;
    const long long nchunks = (rows + oztc::kChunk - 1) / oztc::kChunk;
    int nb = (int)std::min<long long>(std::min<long long>(nblk, oztc::sm_count()), nchunks);
    if (nb < 1) nb = 1;
    const size_t smem = std::max(oztc::GramGeo(m, W != nullptr).smem(), oztc::kMinSmem);
    oztc::gram_tc_kernel<<<nb, oztc::kGThreads, smem, st>>>(Y, W, rows, ld, col0, m, partial, err);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_sum_partials_herm(partial, nb, m, W ? 2 : 1, out, st);
}

cudaError_t launch_rotate_tc(const double2* Y, const double2* W, int ld, int col0, int m, const double2* Q, int mq,
                             const double* theta, double2* X, double2* HX, long long rows, double* res_partial,
                             int nblk, double* res_out, int* err, cudaStream_t st) {
    if (!tc_supported(m, mq) || !err || (!W) != (!HX)) return cudaErrorInvalidValue;
    const long long ntiles = (rows + oztc::kChunk - 1) / oztc::kChunk;
    int nb = (int)std::min<long long>(std::min<long long>(nblk, oztc::sm_count()), ntiles);
    if (nb < 1) nb = 1;
    const bool want_res = theta && W && res_partial && res_out;
    const size_t smem = std::max(oztc::RotGeo(m, mq).smem(), oztc::kMinSmem);
    oztc::rotate_tc_kernel<<<nb, oztc::kRThreads, smem, st>>>(Y, W, ld, col0, m, Q, mq, want_res ? theta : nullptr, X,
                                                             HX, rows, want_res ? res_partial : nullptr, err);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || !want_res) return e;
    return launch_residual_finish(res_partial, nb, mq, res_out, st);
}

}  // namespace khp
