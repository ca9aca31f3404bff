// Matrix-free 19-point stencil of the discretised 6x6 k.p hole Hamiltonian
// (H_DKK + H_SOI + H'_PB + V of the paper's Eqs. 5-6a on the uniform grid of
// Sec. II B), fused with the three-term Chebyshev recurrence, plus the
// per-point field set-up (on-site matrices, Peierls phases) and the
// Gershgorin upper bound of the spectrum.
//
// Vector blocks are row-major [6*Np][ld] interleaved complex.  One thread
// computes one grid point for VG consecutive vectors: it loads the point's
// 6 x VG values, the 18 neighbours' values (pairs +delta/-delta share one
// real symmetric 3x3 orbital matrix, so the two neighbour values are summed
// first), and writes y = alpha*(H x) + beta*x + gamma*prev.
#include <cuda.h>

#include <cmath>
#include <cstdlib>
#include <cstring>
#include <type_traits>
#include <vector>

#include "khp_common.cuh"
#include "khp_internal.h"

namespace khp {

__device__ __forceinline__ bool inr(int i, int n) { return (unsigned)i < (unsigned)n; }

// Complex updates with a real coefficient.  For FP32 each is one packed
// FP32x2 instruction (fma/add/sub .rn.f32x2, sm_100 and later) acting on
// (re, im); every lane rounds exactly like the scalar .rn instruction.
__device__ __forceinline__ unsigned long long pk(float a, float b) {
    unsigned long long r;
    asm("mov.b64 %0, {%1,%2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ float2 upk(unsigned long long v) {
    float2 r;
    asm("mov.b64 {%0,%1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(v));
    return r;
}

// acc += m x
template <typename R>
__device__ __forceinline__ void axpy_c(cx_t<R>& acc, R m, cx_t<R> x) {
    if constexpr (sizeof(R) == 4) {
        unsigned long long d;
        asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(pk(x.x, x.y)), "l"(pk(m, m)), "l"(pk(acc.x, acc.y)));
        acc = upk(d);
    } else {
        acc.x = fma(m, x.x, acc.x);
        acc.y = fma(m, x.y, acc.y);
    }
}

// acc += -i a x  (re += a x.im, im -= a x.re)
template <typename R>
__device__ __forceinline__ void axpy_mi(cx_t<R>& acc, R a, cx_t<R> x) {
    if constexpr (sizeof(R) == 4) {
        unsigned long long d;
        asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(pk(x.y, x.x)), "l"(pk(a, -a)), "l"(pk(acc.x, acc.y)));
        acc = upk(d);
    } else {
        acc.x = fma(a, x.y, acc.x);
        acc.y = fma(-a, x.x, acc.y);
    }
}

template <typename R>
__device__ __forceinline__ cx_t<R> cadd(cx_t<R> a, cx_t<R> b) {
    if constexpr (sizeof(R) == 4) {
        unsigned long long d;
        asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(pk(a.x, a.y)), "l"(pk(b.x, b.y)));
        return upk(d);
    } else {
        return mk<R>(a.x + b.x, a.y + b.y);
    }
}

template <typename R>
__device__ __forceinline__ cx_t<R> csub(cx_t<R> a, cx_t<R> b) {
    if constexpr (sizeof(R) == 4) {
        unsigned long long d;
        asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(pk(a.x, a.y)), "l"(pk(b.x, b.y)));
        return upk(d);
    } else {
        return mk<R>(a.x - b.x, a.y - b.y);
    }
}

template <typename R, int VG>
__device__ __forceinline__ void load_vg(cx_t<R> (&v)[VG], const cx_t<R>* p) {
    if constexpr (VG == 2 && sizeof(R) == 4) {
        const float4 q = __ldg(reinterpret_cast<const float4*>(p));
        v[0] = mk<R>(q.x, q.y);
        v[1] = mk<R>(q.z, q.w);
    } else {
#pragma unroll
        for (int k = 0; k < VG; ++k) v[k] = __ldg(p + k);
    }
}

template <typename R, int VG>
__device__ __forceinline__ void store_vg(cx_t<R>* p, const cx_t<R> (&v)[VG]) {
    if constexpr (VG == 2 && sizeof(R) == 4) {
        *reinterpret_cast<float4*>(p) = make_float4(v[0].x, v[0].y, v[1].x, v[1].y);
    } else {
#pragma unroll
        for (int k = 0; k < VG; ++k) p[k] = v[k];
    }
}

// Streams read or written once per step (prev, the defect source, y): FP32
// blocks go through the evict-first path so the L1 and L2 keep the
// neighbour planes of x.
template <typename R, int VG>
__device__ __forceinline__ void load_vg_once(cx_t<R> (&v)[VG], const cx_t<R>* p) {
    if constexpr (VG == 2 && sizeof(R) == 4) {
        const float4 q = __ldcs(reinterpret_cast<const float4*>(p));
        v[0] = mk<R>(q.x, q.y);
        v[1] = mk<R>(q.z, q.w);
    } else {
        load_vg<R, VG>(v, p);
    }
}

template <typename R, int VG>
__device__ __forceinline__ void store_vg_once(cx_t<R>* p, const cx_t<R> (&v)[VG]) {
    if constexpr (VG == 2 && sizeof(R) == 4) {
        __stcs(reinterpret_cast<float4*>(p), make_float4(v[0].x, v[0].y, v[1].x, v[1].y));
    } else {
        store_vg<R, VG>(p, v);
    }
}

// acc[s*3 + i][v] (+)= sum_j M_ij x[s*3 + j][v] for the NS spins, M real
// symmetric (00,11,22,12,02,01); entries whose bit is clear in nz are
// structurally zero and skipped (warp-uniform branches)
template <typename R, int VG, bool INIT, int NS = 2>
__device__ __forceinline__ void sym3(cx_t<R> (&acc)[6][VG], const R (&M)[6], unsigned nz,
                                     const cx_t<R> (&x)[6][VG]) {
    if (INIT) {
#pragma unroll
        for (int b = 0; b < 3 * NS; ++b)
#pragma unroll
            for (int v = 0; v < VG; ++v) acc[b][v] = mk<R>(R(0), R(0));
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        if (nz & (1u << k)) {
            const R m = M[k];
#pragma unroll
            for (int s = 0; s < NS; ++s)
#pragma unroll
                for (int v = 0; v < VG; ++v) axpy_c<R>(acc[3 * s + k][v], m, x[3 * s + k][v]);
        }
    }
    // off-diagonal (i, j): 3 -> (1,2), 4 -> (0,2), 5 -> (0,1)
#pragma unroll
    for (int k = 3; k < 6; ++k) {
        if (nz & (1u << k)) {
            const int i = k == 3 ? 1 : 0;
            const int j = k == 5 ? 1 : 2;
            const R m = M[k];
#pragma unroll
            for (int s = 0; s < NS; ++s)
#pragma unroll
                for (int v = 0; v < VG; ++v) {
                    axpy_c<R>(acc[3 * s + i][v], m, x[3 * s + j][v]);
                    axpy_c<R>(acc[3 * s + j][v], m, x[3 * s + i][v]);
                }
        }
    }
}

// Orbitals read through a neighbour pair: orbital j is needed when some
// nonzero entry (i, j) of the pair's symmetric 3x3 exists.
__host__ __device__ constexpr unsigned need_of(unsigned nz) {
    return ((nz & (1u | 16u | 32u)) ? 1u : 0u) | ((nz & (2u | 8u | 32u)) ? 2u : 0u) |
           ((nz & (4u | 8u | 16u)) ? 4u : 0u);
}

// acc[3s+i] += (mc * u[3s+j] + i-part) for entry (i, j):
//   PH_SYM pairs:  m * (c u - i s v)  with u = x+ + x-, v = x+ - x-
//   other pairs:   m * u   (mc = m, ms = 0: v unused)
template <typename R, int VG, bool SYMPH, int NS = 2>
__device__ __forceinline__ void pair_entry(cx_t<R> (&acc)[6][VG], int i, int j, R mc, R ms,
                                           const cx_t<R> (&u)[6][VG], const cx_t<R> (&v)[6][VG]) {
#pragma unroll
    for (int sp = 0; sp < NS; ++sp)
#pragma unroll
        for (int w = 0; w < VG; ++w) {
            cx_t<R>& A = acc[3 * sp + i][w];
            axpy_c<R>(A, mc, u[3 * sp + j][w]);
            if (SYMPH) axpy_mi<R>(A, ms, v[3 * sp + j][w]);
        }
}

// y = alpha (H x) + beta x + gamma prev, with alpha folded into the
// coefficients: on-site (alpha o + beta delta) per point, hop and spin-orbit
// matrices pre-scaled by alpha on the host.
// CUBIC: compile-time sparsity of the crystal frame and of frames rotated
// about a cube axis by 45 degrees (the [110] device frame): face pairs are
// diagonal, the edge pair in the (a, b) plane only couples orbitals a and b.
__host__ __device__ constexpr unsigned cubic_nz(int d) {
    return d < 3 ? 7u : (d < 5 ? 32u : (d < 7 ? 16u : 8u));
}

// NB: bands per point, 6 (the spin-orbit k.p Hamiltonian) or 3 (the
// spin-independent H0 block: one spin, no spin-orbit or Zeeman term)
template <typename R, int VG, int PH, bool MASK, bool CUBIC, bool SRC = false, int LD = 0, int MINB = 1, int NB = 6>
__global__ void __launch_bounds__(256, MINB) stencil_kernel(const StencilArgs<R> a) {
    using C = cx_t<R>;
    constexpr int NS = NB / 3;
    const int G = a.ncol / VG;
    const long long np = (long long)a.nx * a.ny * a.nz;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= np * G) return;
    const int g = (int)(t % G);
    const long long p = t / G;
    const int ix = (int)(p % a.nx);
    const long long q = p / a.nx;
    const int iy = (int)(q % a.ny);
    const int iz = (int)(q / a.ny);
    const int ld = LD ? LD : a.ld;              // complex elements per row (compile-time when LD > 0)
    const long long ps = (long long)NB * ld;              // complex elements per point
    const int col = a.col0 + g * VG;
    C* yp = a.y + p * ps + col;

    if (MASK && a.mask[p] == 0) {
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            C z[VG];
#pragma unroll
            for (int v = 0; v < VG; ++v) z[v] = mk<R>(R(0), R(0));
            store_vg<R, VG>(yp + b * ld, z);
        }
        return;
    }

    const C* xp = a.x + p * ps + col;
    C acc[6][VG];
    // acc starts as gamma prev (+ src_coef[col] src): these streams are
    // loaded first, so their latency overlaps the centre and neighbour loads
    // instead of trailing the neighbour sums
    {
        const C* pp = a.prev ? a.prev + p * ps + col : nullptr;
        C pv[6][VG], sv[6][VG];
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            if (pp) load_vg_once<R, VG>(pv[b], pp + b * ld);
            if (SRC) load_vg_once<R, VG>(sv[b], a.src + p * ps + col + b * ld);
        }
        R sc[VG];
        if (SRC) {
#pragma unroll
            for (int v = 0; v < VG; ++v) sc[v] = a.src_coef[col + v];
        }
#pragma unroll
        for (int b = 0; b < NB; ++b)
#pragma unroll
            for (int v = 0; v < VG; ++v) {
                C o = mk<R>(R(0), R(0));
                if (pp) axpy_c<R>(o, a.gamma, pv[b][v]);
                if (SRC) axpy_c<R>(o, sc[v], sv[b][v]);
                acc[b][v] = o;
            }
    }
    {
        C xs[6][VG];
#pragma unroll
        for (int b = 0; b < NB; ++b) load_vg<R, VG>(xs[b], xp + b * ld);
        R o[6];
#pragma unroll
        for (int k = 0; k < 6; ++k) o[k] = a.alpha * __ldg(a.onsite + p * 6 + k);
#pragma unroll
        for (int k = 0; k < 3; ++k) o[k] += a.beta;
        sym3<R, VG, false, NS>(acc, o, a.c.onsite_nz | 7u, xs);
        // spin-orbit + Zeeman (alpha-scaled): constant complex 6x6, zero parts skipped
#pragma unroll
        for (int b = 0; b < (NB == 6 ? 6 : 0); ++b) {
            const unsigned rowm = a.c.soz_nz[b];
#pragma unroll
            for (int b2 = 0; b2 < 6; ++b2) {
                if (rowm & (1u << (2 * b2))) {
                    const R sr = a.c.soz_re[b][b2];
#pragma unroll
                    for (int v = 0; v < VG; ++v) axpy_c<R>(acc[b][v], sr, xs[b2][v]);
                }
                if (rowm & (2u << (2 * b2))) {
                    const R si = a.c.soz_im[b][b2];
#pragma unroll
                    for (int v = 0; v < VG; ++v) axpy_mi<R>(acc[b][v], -si, xs[b2][v]);
                }
            }
        }
    }

#pragma unroll
    for (int d = 0; d < 9; ++d) {
        const unsigned nzd = CUBIC ? cubic_nz(d) : a.c.hop_nz[d];
        if (nzd == 0) continue;
        const unsigned need = need_of(nzd);
        const int dx = pair_dx(d), dy = pair_dy(d), dz = pair_dz(d);
        const long long off = (long long)dx + (long long)a.nx * ((long long)dy + (long long)a.ny * dz);
        const bool inp = inr(ix + dx, a.nx) && inr(iy + dy, a.ny) && inr(iz + dz, a.nz);
        const bool inm = inr(ix - dx, a.nx) && inr(iy - dy, a.ny) && inr(iz - dz, a.nz);
        // neighbour addresses are clamped to this point's own row when the
        // neighbour lies outside the grid, so that every address formed is
        // inside the block even if a load is issued ahead of its predicate
        const long long offp = inp ? off : 0, offm = inm ? off : 0;
        bool okp = inp, okm = inm;
        if (MASK) {
            okp = okp && a.mask[p + offp] != 0;
            okm = okm && a.mask[p - offm] != 0;
        }
        const bool ph = PH != PH_NONE && (a.c.pair_phase & (1u << d));
        const C* xpp = xp + offp * ps;
        const C* xpm = xp - offm * ps;
        C u[6][VG], w[6][VG];
        if (PH == PH_GEN && ph) {
            // general gauge: s = e1 x+ + e2 x- formed per needed component
            const C e1 = __ldg(a.phase + p * 18 + 2 * d);
            const C e2 = __ldg(a.phase + p * 18 + 2 * d + 1);
#pragma unroll
            for (int o = 0; o < 3; ++o) {
                if (!(need & (1u << o))) continue;
#pragma unroll
                for (int sp = 0; sp < NS; ++sp) {
                    const int b = 3 * sp + o;
                    C xpv[VG], xmv[VG];
                    if (okp) load_vg<R, VG>(xpv, xpp + b * ld);
                    else {
#pragma unroll
                        for (int v = 0; v < VG; ++v) xpv[v] = mk<R>(R(0), R(0));
                    }
                    if (okm) load_vg<R, VG>(xmv, xpm + b * ld);
                    else {
#pragma unroll
                        for (int v = 0; v < VG; ++v) xmv[v] = mk<R>(R(0), R(0));
                    }
#pragma unroll
                    for (int v = 0; v < VG; ++v) {
                        u[b][v] = cmul(e1, xpv[v]);
                        cfma(u[b][v], e2, xmv[v]);
                    }
                }
            }
        } else {
#pragma unroll
            for (int o = 0; o < 3; ++o) {
                if (!(need & (1u << o))) continue;
#pragma unroll
                for (int sp = 0; sp < NS; ++sp) {
                    const int b = 3 * sp + o;
                    C xpv[VG], xmv[VG];
                    if (okp) load_vg<R, VG>(xpv, xpp + b * ld);
                    else {
#pragma unroll
                        for (int v = 0; v < VG; ++v) xpv[v] = mk<R>(R(0), R(0));
                    }
                    if (okm) load_vg<R, VG>(xmv, xpm + b * ld);
                    else {
#pragma unroll
                        for (int v = 0; v < VG; ++v) xmv[v] = mk<R>(R(0), R(0));
                    }
#pragma unroll
                    for (int v = 0; v < VG; ++v) {
                        u[b][v] = cadd<R>(xpv[v], xmv[v]);
                        if (PH == PH_SYM && ph) w[b][v] = csub<R>(xpv[v], xmv[v]);
                    }
                }
            }
        }
        // fold the pair's (alpha-scaled) matrix into the phase factors
        R cth = R(1), sth = R(0);
        if (PH == PH_SYM && ph) {
            const C cs = __ldg(a.phase + p * 9 + d);
            cth = cs.x;
            sth = cs.y;
        }
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            if (!(nzd & (1u << k))) continue;
            const R m = a.c.hop[d][k];
            const int i = k < 3 ? k : (k == 3 ? 1 : 0);
            const int j = k < 3 ? k : (k == 5 ? 1 : 2);
            if (PH == PH_SYM && ph) {
                const R mc = m * cth, ms = m * sth;
                pair_entry<R, VG, true, NS>(acc, i, j, mc, ms, u, w);
                if (k >= 3) pair_entry<R, VG, true, NS>(acc, j, i, mc, ms, u, w);
            } else {
                pair_entry<R, VG, false, NS>(acc, i, j, m, R(0), u, w);
                if (k >= 3) pair_entry<R, VG, false, NS>(acc, j, i, m, R(0), u, w);
            }
        }
    }

#pragma unroll
    for (int b = 0; b < NB; ++b) store_vg_once<R, VG>(yp + b * ld, acc[b]);
}

template <typename R, int VG, int PH>
static cudaError_t launch_ph(const StencilArgs<R>& a, unsigned blocks, cudaStream_t st) {
    bool cubic = true;
    for (int d = 0; d < 9; ++d) cubic = cubic && (a.c.hop_nz[d] & ~cubic_nz(d)) == 0;
    if (a.nb == 3) {
        // spin-independent H0: no magnetic field, so no Peierls phases
        if constexpr (PH == PH_NONE) {
            if (a.src) {
                if constexpr (sizeof(R) == 8) return cudaErrorNotSupported;
                if (a.mask) {
                    if (cubic) stencil_kernel<R, VG, PH, true, true, true, 0, 1, 3><<<blocks, 256, 0, st>>>(a);
                    else stencil_kernel<R, VG, PH, true, false, true, 0, 1, 3><<<blocks, 256, 0, st>>>(a);
                } else {
                    if (cubic) stencil_kernel<R, VG, PH, false, true, true, 0, 1, 3><<<blocks, 256, 0, st>>>(a);
                    else stencil_kernel<R, VG, PH, false, false, true, 0, 1, 3><<<blocks, 256, 0, st>>>(a);
                }
            } else {
                if (a.mask) {
                    if (cubic) stencil_kernel<R, VG, PH, true, true, false, 0, 1, 3><<<blocks, 256, 0, st>>>(a);
                    else stencil_kernel<R, VG, PH, true, false, false, 0, 1, 3><<<blocks, 256, 0, st>>>(a);
                } else {
                    if (cubic) stencil_kernel<R, VG, PH, false, true, false, 0, 1, 3><<<blocks, 256, 0, st>>>(a);
                    else stencil_kernel<R, VG, PH, false, false, false, 0, 1, 3><<<blocks, 256, 0, st>>>(a);
                }
            }
            return cudaGetLastError();
        } else {
            return cudaErrorNotSupported;
        }
    }
    if constexpr (VG == 2) {
        if (cubic && !a.mask) {
            // hot path: row length known at compile time (immediate band offsets)
#define KHP_LD_CASE(L)                                                                               \
            if (a.ld == L) {                                                                         \
                if constexpr (sizeof(R) == 4) {                                                      \
                    if (a.src) stencil_kernel<R, VG, PH, false, true, true, L, 2><<<blocks, 256, 0, st>>>(a); \
                    else stencil_kernel<R, VG, PH, false, true, false, L, 2><<<blocks, 256, 0, st>>>(a);      \
                } else {                                                                             \
                    if (a.src) return cudaErrorNotSupported;                                         \
                    stencil_kernel<R, VG, PH, false, true, false, L, 1><<<blocks, 256, 0, st>>>(a);  \
                }                                                                                    \
                return cudaGetLastError();                                                           \
            }
            KHP_LD_CASE(16)
            KHP_LD_CASE(20)
            KHP_LD_CASE(24)
            KHP_LD_CASE(32)
#undef KHP_LD_CASE
        }
    }
    if constexpr (sizeof(R) == 4) {
        if (a.src) {
            // defect-corrected FP32 filter steps
            if (a.mask) {
                if (cubic) stencil_kernel<R, VG, PH, true, true, true><<<blocks, 256, 0, st>>>(a);
                else stencil_kernel<R, VG, PH, true, false, true><<<blocks, 256, 0, st>>>(a);
            } else {
                if (cubic) stencil_kernel<R, VG, PH, false, true, true><<<blocks, 256, 0, st>>>(a);
                else stencil_kernel<R, VG, PH, false, false, true><<<blocks, 256, 0, st>>>(a);
            }
            return cudaGetLastError();
        }
    } else {
        if (a.src) return cudaErrorNotSupported;
    }
    if (a.mask) {
        if (cubic) stencil_kernel<R, VG, PH, true, true><<<blocks, 256, 0, st>>>(a);
        else stencil_kernel<R, VG, PH, true, false><<<blocks, 256, 0, st>>>(a);
    } else {
        if (cubic) stencil_kernel<R, VG, PH, false, true><<<blocks, 256, 0, st>>>(a);
        else stencil_kernel<R, VG, PH, false, false><<<blocks, 256, 0, st>>>(a);
    }
    return cudaGetLastError();
}

template <typename R, int VG>
static cudaError_t launch_vg(const StencilArgs<R>& a, cudaStream_t st) {
    const long long np = (long long)a.nx * a.ny * a.nz;
    const long long total = np * (a.ncol / VG);
    if (total == 0) return cudaSuccess;
    const int threads = 256;
    const long long blocks = (total + threads - 1) / threads;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    const int mode = a.phase ? a.phase_mode : PH_NONE;
    if (mode == PH_SYM) return launch_ph<R, VG, PH_SYM>(a, (unsigned)blocks, st);
    if (mode == PH_GEN) return launch_ph<R, VG, PH_GEN>(a, (unsigned)blocks, st);
    return launch_ph<R, VG, PH_NONE>(a, (unsigned)blocks, st);
}

template <typename R>
cudaError_t launch_stencil(const StencilArgs<R>& a, cudaStream_t st) {
    if constexpr (sizeof(R) == 4) {
        const cudaError_t e = launch_stencil_plane(a, a.err, st);
        if (e != cudaErrorNotSupported) return e;
    }
    if ((a.ncol % 2) == 0 && (a.col0 % 2) == 0 && (a.ld % 2) == 0) return launch_vg<R, 2>(a, st);
    return launch_vg<R, 1>(a, st);
}

template cudaError_t launch_stencil<double>(const StencilArgs<double>&, cudaStream_t);
template cudaError_t launch_stencil<float>(const StencilArgs<float>&, cudaStream_t);

// ------------------------------------------- plane-marching FP32 stencil
// The same fused step y = alpha (H x) + beta x + gamma prev + c_col src for
// FP32 blocks, organised for data reuse: a CTA owns an x-y tile of
// 16 x 4 points and V = 4 vector columns (one per thread) and marches
// through a range of z-planes.  The planes of x, each with a one-point halo
// in x and y, arrive in a four-deep shared-memory ring by TMA
// (cp.async.bulk.tensor, one box per band, so a band of a plane is a dense
// [y][x][col] array read without bank conflicts); the box reads zeros
// outside the grid, which is the Dirichlet wall.  prev and the defect
// source arrive by TMA as well, one plane ahead of their use.  All 19
// neighbour values come from shared memory, and every byte of x, prev and
// src crosses HBM once (the halo is re-read from L2).  Three warps issue
// the copies (x, prev, src); each copy completes on an mbarrier; one CTA
// barrier per plane releases the buffers.  Every wait is bounded (about a
// second): a wait that runs out sets bit 8 of the error flag, and the CTA
// waits (bounded) for its copies in flight and leaves.
namespace plane {

constexpr int TX = 16;
constexpr int V = 4;
constexpr int HX = TX + 2;

// NSX: depth of the ring of x planes (4: plane z + 3 is loaded while plane z
// is computed; 3: plane z + 2 is loaded into the slot of plane z - 1 as soon
// as the pairs that reach across planes are summed).  NPS: buffers of the
// prev/src planes (2: the plane after next is loaded while a plane is
// computed).
template <int NB, int TY, int NSX, int NPS, int VG>
struct Geo {
    static constexpr int HY = TY + 2;
    static constexpr int THREADS = TX * TY * V / VG;
    static constexpr int CTAS_PER_SM = 512 / (TX * TY * V);   // by shared memory (ring 4: 2 at TY = 4)
    static constexpr int XBAND = HY * HX * V;           // float2 per band of a halo plane
    static constexpr int XSLOT = NB * XBAND;
    static constexpr int PBAND = TY * TX * V;           // float2 per band of a prev/src plane
    static constexpr int PPLANE = NB * PBAND;
    static constexpr int NBAR = NSX + NPS;
    static constexpr int SMEM = (NSX * XSLOT + 2 * NPS * PPLANE) * 8 + 8 * NBAR;
};

struct Work {
    int ntx, nty, ngroups, zch, nzc;
    int cbase;                 // first column of group 0 (even)
    int* err;                  // bit 8 set when a pipeline wait runs out
};

__device__ __forceinline__ uint32_t sa(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

// Bounded wait for the phase with the given parity: false after ~2^31 cycles.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    const long long t0 = clock64();
    while (true) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred P;\n mbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2;\n selp.u32 %0, 1, 0, P;\n}"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
        if (clock64() - t0 > (1LL << 31)) return false;
    }
}

__device__ __forceinline__ void tma_load5(uint32_t dst, const CUtensorMap* map, int c0, int c1, int c2, int c3, int c4,
                                          uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(dst),
        "l"(reinterpret_cast<unsigned long long>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(bar)
        : "memory");
}

// One work item (column group, tile, z-chunk) of one step; a, w and the
// maps live in the kernel's parameter space (grid constants).
template <int NB, int PH, bool SRC, int TY, int NSX, int NPS, int VG>
__device__ __forceinline__ void plane_item(const StencilArgs<float>& a, const Work& w, const CUtensorMap& mx,
                                           const CUtensorMap& mp, const CUtensorMap& ms, int item0) {
    using G = Geo<NB, TY, NSX, NPS, VG>;
    using C = float2;
    constexpr int NS = NB / 3;
    static_assert(G::THREADS >= 96, "three issuing warps");
    extern __shared__ __align__(1024) unsigned char smem[];
    C* xring = reinterpret_cast<C*>(smem);
    C* pbuf = xring + NSX * G::XSLOT;             // [NPS][PPLANE]
    C* sbuf = pbuf + NPS * G::PPLANE;             // [NPS][PPLANE]
    unsigned long long* bars = reinterpret_cast<unsigned long long*>(sbuf + NPS * G::PPLANE);

    // work item: column group fastest, so the groups of one tile run together
    int item = item0;
    const int g = item % w.ngroups;
    item /= w.ngroups;
    const int txi = item % w.ntx;
    item /= w.ntx;
    const int tyi = item % w.nty;
    const int zc = item / w.nty;
    const int tx0 = txi * TX, ty0 = tyi * TY;
    const int z0 = zc * w.zch;
    const int zlast = min(z0 + w.zch, a.nz) - 1;
    const int zs = z0 - 1;                      // first plane of the ring
    const int cg = w.cbase + g * V;             // first column of this group

    // thread: VG consecutive columns (from col) of one point (lx, ly)
    constexpr int NCP = V / VG;
    const int tid = threadIdx.x;
    const int col = (tid % NCP) * VG;
    const int lx = (tid / NCP) % TX;
    const int ly = tid / (NCP * TX);
    const int gx = tx0 + lx, gy = ty0 + ly;
    const int c = cg + col;
    const bool live = gx < a.nx && gy < a.ny;
    bool store[VG];
#pragma unroll
    for (int v = 0; v < VG; ++v) store[v] = live && c + v >= a.col0 && c + v < a.col0 + a.ncol;
    const bool has_prev = a.prev != nullptr;
    const bool has_ps = has_prev || SRC;
    const long long plane_pts = (long long)a.nx * a.ny;
    const long long ps = (long long)NB * a.ld;  // complex per point
    // copies are issued by lane 0 of warp 0 (x), warp 1 (prev) and warp 2 (src)
    const bool ix_thread = tid == 0;
    const bool ip_thread = tid == 32 && has_prev;
    const bool is_thread = tid == 64 && SRC;

    // q >= zs always: unsigned division by the compile-time ring sizes
    auto xslot = [&](int q) { return (int)((unsigned)(q - zs) % (unsigned)NSX); };
    auto xpar = [&](int q) { return (uint32_t)(((unsigned)(q - zs) / (unsigned)NSX) & 1u); };
    auto pslot = [&](int q) { return (int)((unsigned)(q - z0) % (unsigned)NPS); };
    auto ppar = [&](int q) { return (uint32_t)(((unsigned)(q - z0) / (unsigned)NPS) & 1u); };
    auto xbar = [&](int q) { return sa(bars + xslot(q)); };
    auto pbar = [&](int q) { return sa(bars + NSX + pslot(q)); };

    auto issue_x = [&](int q) {          // plane q into its ring slot
        const uint32_t bar = xbar(q);
        mbar_expect(bar, G::XSLOT * 8);
#pragma unroll
        for (int b = 0; b < NB; ++b)
            tma_load5(sa(xring + xslot(q) * G::XSLOT + b * G::XBAND), &mx, 2 * cg, b, tx0 - 1, ty0 - 1, q, bar);
    };
    auto issue_p = [&](int q, const CUtensorMap* map, C* buf) {   // one prev/src plane
        const uint32_t bar = pbar(q);
        mbar_expect(bar, G::PPLANE * 8);
#pragma unroll
        for (int b = 0; b < NB; ++b)
            tma_load5(sa(buf + pslot(q) * G::PPLANE + b * G::PBAND), map, 2 * cg, b, tx0, ty0, q, bar);
    };

    if (tid == 0) {
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<unsigned long long>(&mx)) : "memory");
        for (int s = 0; s < NSX; ++s) mbar_init(sa(bars + s), 1);
        for (int s = 0; s < NPS; ++s) mbar_init(sa(bars + NSX + s), (has_prev ? 1 : 0) + (SRC ? 1 : 0));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    // prologue: the first NSX planes of x and NPS planes of prev/src
    const int x_first_last = min(zs + NSX - 1, zlast + 1);
    const int p_first_last = min(z0 + NPS - 1, zlast);
    if (ix_thread)
        for (int q = zs; q <= x_first_last; ++q) issue_x(q);
    if (ip_thread)
        for (int q = z0; q <= p_first_last; ++q) issue_p(q, &mp, pbuf);
    if (is_thread)
        for (int q = z0; q <= p_first_last; ++q) issue_p(q, &ms, sbuf);
    int issued_x = x_first_last, issued_p = has_ps ? p_first_last : z0 - 1;
    int waited_x = zs - 1, waited_p = z0 - 1;

    // per-point fields of the current plane (prefetched one plane ahead)
    auto load_fields = [&](int z, float (&o)[6], float2 (&cs)[9]) {
#pragma unroll
        for (int k = 0; k < 6; ++k) o[k] = 0.f;
#pragma unroll
        for (int d = 0; d < 9; ++d) cs[d] = make_float2(1.f, 0.f);
        if (!live || z > zlast) return;
        const long long p = gx + (long long)a.nx * gy + plane_pts * z;
#pragma unroll
        for (int k = 0; k < 6; ++k) o[k] = __ldg(a.onsite + p * 6 + k);
        if (PH == PH_SYM) {
#pragma unroll
            for (int d = 0; d < 9; ++d) cs[d] = __ldg(a.phase + p * 9 + d);
        }
    };
    float o_cur[6], o_nxt[6];
    float2 cs_cur[9], cs_nxt[9];
    load_fields(z0, o_cur, cs_cur);

    // this thread's point in a ring slot; the slots of planes z - 1, z, z + 1
    // are set once per step, so every neighbour load is a base plus a
    // compile-time offset
    const C* own = xring + ((ly + 1) * HX + (lx + 1)) * V + col;
    auto lds = [](C (&v)[VG], const C* p) {
        if constexpr (VG == 2) {
            const float4 q = *reinterpret_cast<const float4*>(p);
            v[0] = make_float2(q.x, q.y);
            v[1] = make_float2(q.z, q.w);
        } else {
            v[0] = *p;
        }
    };
    const C* slot_base[3] = {own, own, own};
    auto xat = [&](int q, int b, int dx, int dy) -> const C* {
        return slot_base[q] + b * G::XBAND + (dy * HX + dx) * V;
    };
    // pair d: (x+ + x-) and (x+ - x-) of the needed bands, then the pair's
    // alpha-scaled orbital matrix (times the Peierls phase) into acc
    auto pair = [&](C (&acc)[6][VG], int z, auto dc) {
        constexpr int d = decltype(dc)::value;
        constexpr unsigned nzd = cubic_nz(d);
        constexpr unsigned need = need_of(nzd);
        constexpr int dx = pair_dx(d), dy = pair_dy(d), dz = pair_dz(d);
        // in the symmetric gauge every pair takes the phase path (pairs
        // without a phase carry (1, 0)): no runtime branch in the body, so
        // the shared-memory loads of later pairs can be scheduled early
        constexpr bool ph = PH == PH_SYM;
        C u[6][VG], v[6][VG];
#pragma unroll
        for (int o = 0; o < 3; ++o) {
            if (!(need & (1u << o))) continue;
#pragma unroll
            for (int sp = 0; sp < NS; ++sp) {
                const int b = 3 * sp + o;
                C xp[VG], xm[VG];
                lds(xp, xat(1 + dz, b, dx, dy));
                lds(xm, xat(1 - dz, b, -dx, -dy));
#pragma unroll
                for (int t = 0; t < VG; ++t) {
                    u[b][t] = cadd<float>(xp[t], xm[t]);
                    if (PH == PH_SYM) v[b][t] = csub<float>(xp[t], xm[t]);
                }
            }
        }
        float cth = 1.f, sth = 0.f;
        if (PH == PH_SYM && ph) {
            cth = cs_cur[d].x;
            sth = cs_cur[d].y;
        }
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            if (!(nzd & (1u << k))) continue;
            const float m = a.c.hop[d][k];
            const int i = k < 3 ? k : (k == 3 ? 1 : 0);
            const int j = k < 3 ? k : (k == 5 ? 1 : 2);
            if (PH == PH_SYM && ph) {
                const float mc = m * cth, msn = m * sth;
                pair_entry<float, VG, true, NS>(acc, i, j, mc, msn, u, v);
                if (k >= 3) pair_entry<float, VG, true, NS>(acc, j, i, mc, msn, u, v);
            } else {
                pair_entry<float, VG, false, NS>(acc, i, j, m, 0.f, u, v);
                if (k >= 3) pair_entry<float, VG, false, NS>(acc, j, i, m, 0.f, u, v);
            }
        }
    };

    bool failed = false;
    for (int z = z0; z <= zlast; ++z) {
        // planes z - 1 .. z + 1 of x (one new plane per step after the first)
        for (int q = waited_x + 1; q <= z + 1; ++q) failed |= !mbar_wait(xbar(q), xpar(q));
        waited_x = z + 1;
        load_fields(z + 1, o_nxt, cs_nxt);
#pragma unroll
        for (int k = 0; k < 3; ++k) slot_base[k] = own + xslot(z - 1 + k) * G::XSLOT;

        C acc[6][VG];
#pragma unroll
        for (int b = 0; b < 6; ++b)
#pragma unroll
            for (int t = 0; t < VG; ++t) acc[b][t] = make_float2(0.f, 0.f);
        // the pairs that reach planes z - 1 and z + 1 first
        pair(acc, z, std::integral_constant<int, 2>{});
        pair(acc, z, std::integral_constant<int, 5>{});
        pair(acc, z, std::integral_constant<int, 6>{});
        pair(acc, z, std::integral_constant<int, 7>{});
        pair(acc, z, std::integral_constant<int, 8>{});
        if (NSX == 3) {
            // plane z - 1 is done with: plane z + 2 goes into its slot
            __syncthreads();
            if (ix_thread && z + 2 <= zlast + 1) {
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                issue_x(z + 2);
            }
            if (z + 2 <= zlast + 1) issued_x = z + 2;
        }
        // centre: on-site orbital matrix (+ beta), spin-orbit and Zeeman;
        // all entries are applied (zeros add nothing), with no runtime branch
        {
            C xs[6][VG];
#pragma unroll
            for (int b = 0; b < NB; ++b) lds(xs[b], xat(1, b, 0, 0));
            float oo[6];
#pragma unroll
            for (int k = 0; k < 6; ++k) oo[k] = a.alpha * o_cur[k];
#pragma unroll
            for (int k = 0; k < 3; ++k) oo[k] += a.beta;
            sym3<float, VG, false, NS>(acc, oo, 63u, xs);
#pragma unroll
            for (int b = 0; b < (NB == 6 ? 6 : 0); ++b)
#pragma unroll
                for (int b2 = 0; b2 < 6; ++b2)
#pragma unroll
                    for (int t = 0; t < VG; ++t) {
                        axpy_c<float>(acc[b][t], a.c.soz_re[b][b2], xs[b2][t]);
                        axpy_mi<float>(acc[b][t], -a.c.soz_im[b][b2], xs[b2][t]);
                    }
        }
        // the pairs inside plane z
        pair(acc, z, std::integral_constant<int, 0>{});
        pair(acc, z, std::integral_constant<int, 1>{});
        pair(acc, z, std::integral_constant<int, 3>{});
        pair(acc, z, std::integral_constant<int, 4>{});

        // gamma prev + c_col src
        if (has_ps) {
            failed |= !mbar_wait(pbar(z), ppar(z));
            waited_p = z;
            const int pi = pslot(z) * G::PPLANE + (ly * TX + lx) * V + col;
            float sc[VG];
#pragma unroll
            for (int t = 0; t < VG; ++t) sc[t] = SRC ? a.src_coef[min(max(c + t, 0), 63)] : 0.f;
#pragma unroll
            for (int b = 0; b < NB; ++b) {
                C pv[VG], sv[VG];
                if (has_prev) lds(pv, pbuf + pi + b * G::PBAND);
                if (SRC) lds(sv, sbuf + pi + b * G::PBAND);
#pragma unroll
                for (int t = 0; t < VG; ++t) {
                    if (has_prev) axpy_c<float>(acc[b][t], a.gamma, pv[t]);
                    if (SRC) axpy_c<float>(acc[b][t], sc[t], sv[t]);
                }
            }
        }
        {
            C* yp = a.y + (gx + (long long)a.nx * gy + plane_pts * z) * ps + c;
            if (VG == 2 && store[0] && store[VG - 1]) {
#pragma unroll
                for (int b = 0; b < NB; ++b)
                    __stcs(reinterpret_cast<float4*>(yp + b * a.ld),
                           make_float4(acc[b][0].x, acc[b][0].y, acc[b][VG - 1].x, acc[b][VG - 1].y));
            } else {
#pragma unroll
                for (int t = 0; t < VG; ++t)
                    if (store[t])
#pragma unroll
                        for (int b = 0; b < NB; ++b) __stcs(yp + b * a.ld + t, acc[b][t]);
            }
        }
        // every thread is done with this step's buffers; a wait that ran out
        // anywhere ends the CTA (after its copies in flight have landed)
        if (__syncthreads_or(failed)) {
            if (tid == 0) {
                atomicOr(w.err, 8);
                for (int q = waited_x + 1; q <= issued_x; ++q) mbar_wait(xbar(q), xpar(q));
                for (int q = waited_p + 1; q <= issued_p; ++q) mbar_wait(pbar(q), ppar(q));
            }
            return;
        }
        const bool more_p = has_ps && z + NPS <= zlast;
        if (NSX == 4 && ix_thread && z + 3 <= zlast + 1) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            issue_x(z + 3);
        }
        if (more_p && (ip_thread || is_thread)) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            if (ip_thread) issue_p(z + NPS, &mp, pbuf);
            if (is_thread) issue_p(z + NPS, &ms, sbuf);
        }
        if (NSX == 4 && z + 3 <= zlast + 1) issued_x = z + 3;
        if (more_p) issued_p = z + NPS;
#pragma unroll
        for (int k = 0; k < 6; ++k) o_cur[k] = o_nxt[k];
#pragma unroll
        for (int d = 0; d < 9; ++d) cs_cur[d] = cs_nxt[d];
    }
}

template <int NB, int PH, bool SRC, int TY, int NSX, int NPS, int VG>
__global__ void __launch_bounds__(Geo<NB, TY, NSX, NPS, VG>::THREADS, Geo<NB, TY, NSX, NPS, VG>::CTAS_PER_SM)
    stencil_plane_kernel(const __grid_constant__ StencilArgs<float> a, const __grid_constant__ Work w,
                         const __grid_constant__ CUtensorMap mx, const __grid_constant__ CUtensorMap mp,
                         const __grid_constant__ CUtensorMap ms) {
    plane_item<NB, PH, SRC, TY, NSX, NPS, VG>(a, w, mx, mp, ms, blockIdx.x);
}

// The same step of up to KG problems of a batch in one launch: the work
// items of problem q are blocks item0[q] .. item0[q + 1] - 1.
constexpr int KG = 8;
struct GroupParams {
    CUtensorMap mx[KG], mp[KG], ms[KG];
    StencilArgs<float> a[KG];
    Work w[KG];
    int item0[KG + 1];
    int count;
};

template <int NB, int PH, bool SRC, int TY, int NSX, int NPS, int VG>
__global__ void __launch_bounds__(Geo<NB, TY, NSX, NPS, VG>::THREADS, Geo<NB, TY, NSX, NPS, VG>::CTAS_PER_SM)
    stencil_plane_group_kernel(const __grid_constant__ GroupParams gp) {
    int q = 0;
    while (q + 1 < gp.count && (int)blockIdx.x >= gp.item0[q + 1]) ++q;
    plane_item<NB, PH, SRC, TY, NSX, NPS, VG>(gp.a[q], gp.w[q], gp.mx[q], gp.mp[q], gp.ms[q],
                                              (int)blockIdx.x - gp.item0[q]);
}

typedef CUresult (*EncodeTiled)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encoder() {
    static EncodeTiled fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiled>(p);
        else
            cudaGetLastError();
    }
    return fn;
}

// 5-d map of a [nz][ny][nx][nb][ld] complex64 block as floats: dims
// (2 ld, nb, nx, ny, nz), box (2 V, 1, bx, by, 1)
bool make_map(CUtensorMap* m, const void* base, int ld, int nb, int nx, int ny, int nz, int bx, int by) {
    EncodeTiled enc = encoder();
    if (!enc) return false;
    const cuuint64_t dims[5] = {(cuuint64_t)2 * ld, (cuuint64_t)nb, (cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)nz};
    const cuuint64_t row = (cuuint64_t)ld * 8;
    const cuuint64_t strides[4] = {row, row * nb, row * nb * nx, row * nb * nx * ny};
    const cuuint32_t box[5] = {2 * V, 1, (cuuint32_t)bx, (cuuint32_t)by, 1};
    const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 5, const_cast<void*>(base), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// KHP_STENCIL_PLANE=0 in the environment selects the per-point kernel for
// every FP32 step (for comparisons); read once.
bool enabled() {
    static int on = -1;
    if (on < 0) {
        const char* e = std::getenv("KHP_STENCIL_PLANE");
        on = (e && e[0] == '0') ? 0 : 1;
    }
    return on == 1;
}

// The measured best shape on B300 (C2, 24 vectors): tile 16 x 4 points x
// 4 vectors, one vector per thread, x ring of 4 planes, one prev/src plane:
// two 256-thread CTAs per SM.
constexpr int kTY = 4, kNSX = 4, kNPS = 1, kVG = 1;

template <int NB, int PH, bool SRC>
cudaError_t launch_t(const StencilArgs<float>& a, const Work& w, unsigned items, const CUtensorMap& mx,
                     const CUtensorMap& mp, const CUtensorMap& ms, cudaStream_t st) {
    using G = Geo<NB, kTY, kNSX, kNPS, kVG>;
    stencil_plane_kernel<NB, PH, SRC, kTY, kNSX, kNPS, kVG><<<items, G::THREADS, G::SMEM, st>>>(a, w, mx, mp, ms);
    return cudaGetLastError();
}

template <int NB, int PH, bool SRC>
cudaError_t prep_t() {
    return cudaFuncSetAttribute(stencil_plane_kernel<NB, PH, SRC, kTY, kNSX, kNPS, kVG>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, Geo<NB, kTY, kNSX, kNPS, kVG>::SMEM);
}

}  // namespace plane


namespace plane {

// Work split and tensor maps of one step; cudaErrorNotSupported when the
// plane kernel does not cover it (FP32 only: no mask, the crystal or [110]
// frame, B = 0 or the symmetric gauge, even row length and first column).
cudaError_t prepare(const StencilArgs<float>& a, int* err, Work* w, CUtensorMap* mx, CUtensorMap* mp,
                    CUtensorMap* ms, int* mode, long long* items) {
    if (!enabled() || a.mask || (a.ld & 1) || (a.col0 & 1) || a.ncol < 1 || !err) return cudaErrorNotSupported;
    if (a.nb != 6 && a.nb != 3) return cudaErrorNotSupported;
    bool cubic = true;
    for (int d = 0; d < 9; ++d) cubic = cubic && (a.c.hop_nz[d] & ~cubic_nz(d)) == 0;
    if (!cubic) return cudaErrorNotSupported;
    *mode = a.phase ? a.phase_mode : PH_NONE;
    if (*mode == PH_GEN || (a.nb == 3 && *mode != PH_NONE)) return cudaErrorNotSupported;
    const int per_sm = Geo<6, kTY, kNSX, kNPS, kVG>::CTAS_PER_SM;
    w->ntx = (a.nx + TX - 1) / TX;
    w->nty = (a.ny + kTY - 1) / kTY;
    w->cbase = a.col0 & ~1;
    w->ngroups = (a.col0 + a.ncol - w->cbase + V - 1) / V;
    w->err = err;
    int dev = 0, sms = 148;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // z-chunk: the fewest passes over the grid in waves of the resident
    // CTAs; a chunk costs its planes plus about three planes of start-up
    // (its two boundary planes of x and the first copies in flight)
    const long long tiles = (long long)w->ntx * w->nty * w->ngroups;
    int best = a.nz;
    double best_cost = 1e300;
    for (int zch = 4; zch <= a.nz + 3; ++zch) {
        const int zc = std::min(zch, a.nz);
        const long long it = tiles * ((a.nz + zc - 1) / zc);
        const double waves = std::ceil((double)it / (sms * per_sm));
        const double cost = waves * (zc + 3.0);
        if (cost < best_cost - 1e-9) { best_cost = cost; best = zc; }
        if (zch >= a.nz) break;
    }
    w->zch = std::max(1, best);
    w->nzc = (a.nz + w->zch - 1) / w->zch;
    *items = tiles * w->nzc;
    if (*items > 0x7fffffffLL) return cudaErrorNotSupported;
    std::memset(mp, 0, sizeof(*mp));
    std::memset(ms, 0, sizeof(*ms));
    if (!make_map(mx, a.x, a.ld, a.nb, a.nx, a.ny, a.nz, HX, kTY + 2)) return cudaErrorNotSupported;
    if (a.prev && !make_map(mp, a.prev, a.ld, a.nb, a.nx, a.ny, a.nz, TX, kTY)) return cudaErrorNotSupported;
    if (a.src && !make_map(ms, a.src, a.ld, a.nb, a.nx, a.ny, a.nz, TX, kTY)) return cudaErrorNotSupported;
    return cudaSuccess;
}

template <int NB, int PH, bool SRC>
cudaError_t launch_group_t(const GroupParams& gp, unsigned items, cudaStream_t st) {
    using G = Geo<NB, kTY, kNSX, kNPS, kVG>;
    stencil_plane_group_kernel<NB, PH, SRC, kTY, kNSX, kNPS, kVG><<<items, G::THREADS, G::SMEM, st>>>(gp);
    return cudaGetLastError();
}

template <int NB, int PH, bool SRC>
cudaError_t prep_group_t() {
    return cudaFuncSetAttribute(stencil_plane_group_kernel<NB, PH, SRC, kTY, kNSX, kNPS, kVG>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, Geo<NB, kTY, kNSX, kNPS, kVG>::SMEM);
}

}  // namespace plane

cudaError_t launch_stencil_plane(const StencilArgs<float>& a, int* err, cudaStream_t st) {
    using namespace plane;
    if ((long long)a.nx * a.ny * a.nz == 0) return cudaSuccess;
    Work w;
    CUtensorMap mx, mp, ms;
    int mode = PH_NONE;
    long long items = 0;
    const cudaError_t e = prepare(a, err, &w, &mx, &mp, &ms, &mode, &items);
    if (e != cudaSuccess) return e;
    const unsigned n = (unsigned)items;
    if (a.nb == 6) {
        if (mode == PH_SYM)
            return a.src ? launch_t<6, PH_SYM, true>(a, w, n, mx, mp, ms, st)
                         : launch_t<6, PH_SYM, false>(a, w, n, mx, mp, ms, st);
        return a.src ? launch_t<6, PH_NONE, true>(a, w, n, mx, mp, ms, st)
                     : launch_t<6, PH_NONE, false>(a, w, n, mx, mp, ms, st);
    }
    return a.src ? launch_t<3, PH_NONE, true>(a, w, n, mx, mp, ms, st)
                 : launch_t<3, PH_NONE, false>(a, w, n, mx, mp, ms, st);
}

// The same filter step of several problems as grouped launches: the
// problems are partitioned by gauge mode, and each part goes out in
// launches of up to KG problems.  cudaErrorNotSupported, with nothing
// launched, unless the plane kernel covers every step with the same bands
// and source term.
cudaError_t launch_stencil_plane_group(const StencilArgs<float>* const* a, int count, cudaStream_t st) {
    using namespace plane;
    if (count < 1) return cudaSuccess;
    struct Prep {
        Work w;
        CUtensorMap mx, mp, ms;
        int mode;
        long long items;
    };
    std::vector<Prep> pr(count);
    for (int i = 0; i < count; ++i) {
        const StencilArgs<float>& ai = *a[i];
        if ((long long)ai.nx * ai.ny * ai.nz == 0) return cudaErrorNotSupported;
        const cudaError_t e = prepare(ai, ai.err, &pr[i].w, &pr[i].mx, &pr[i].mp, &pr[i].ms, &pr[i].mode,
                                      &pr[i].items);
        if (e != cudaSuccess) return e;
        if (ai.nb != a[0]->nb || (ai.src != nullptr) != (a[0]->src != nullptr)) return cudaErrorNotSupported;
    }
    const bool src = a[0]->src != nullptr;
    GroupParams gp;
    for (int mode : {PH_NONE, PH_SYM}) {
        int q = 0;
        long long total = 0;
        auto flush = [&]() -> cudaError_t {
            if (q == 0) return cudaSuccess;
            gp.count = q;
            gp.item0[q] = (int)total;
            const unsigned n = (unsigned)total;
            cudaError_t e;
            if (a[0]->nb == 6) {
                if (mode == PH_SYM)
                    e = src ? launch_group_t<6, PH_SYM, true>(gp, n, st) : launch_group_t<6, PH_SYM, false>(gp, n, st);
                else
                    e = src ? launch_group_t<6, PH_NONE, true>(gp, n, st) : launch_group_t<6, PH_NONE, false>(gp, n, st);
            } else {
                e = src ? launch_group_t<3, PH_NONE, true>(gp, n, st) : launch_group_t<3, PH_NONE, false>(gp, n, st);
            }
            q = 0;
            total = 0;
            return e;
        };
        for (int i = 0; i < count; ++i) {
            if (pr[i].mode != mode) continue;
            if (q == KG || total + pr[i].items > 0x7fffffffLL) {
                const cudaError_t e = flush();
                if (e != cudaSuccess) return e;
            }
            gp.a[q] = *a[i];
            gp.w[q] = pr[i].w;
            gp.mx[q] = pr[i].mx;
            gp.mp[q] = pr[i].mp;
            gp.ms[q] = pr[i].ms;
            gp.item0[q] = (int)total;
            total += pr[i].items;
            ++q;
        }
        const cudaError_t e = flush();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t prepare_plane() {
    using namespace plane;
    cudaError_t e = prep_t<6, PH_NONE, false>();
    if (e == cudaSuccess) e = prep_t<6, PH_NONE, true>();
    if (e == cudaSuccess) e = prep_t<6, PH_SYM, false>();
    if (e == cudaSuccess) e = prep_t<6, PH_SYM, true>();
    if (e == cudaSuccess) e = prep_t<3, PH_NONE, false>();
    if (e == cudaSuccess) e = prep_t<3, PH_NONE, true>();
    if (e == cudaSuccess) e = prep_group_t<6, PH_NONE, false>();
    if (e == cudaSuccess) e = prep_group_t<6, PH_NONE, true>();
    if (e == cudaSuccess) e = prep_group_t<6, PH_SYM, false>();
    if (e == cudaSuccess) e = prep_group_t<6, PH_SYM, true>();
    if (e == cudaSuccess) e = prep_group_t<3, PH_NONE, false>();
    if (e == cudaSuccess) e = prep_group_t<3, PH_NONE, true>();
    return e;
}

// ------------------------------------------------------------ field set-up
struct FieldArgs {
    int nx, ny, nz;
    const double* V;
    const double* strain;     // [6][np] or null
    const double* levers;     // [ng][np] or null
    int ng;
    double alpha[KHP_MAX_GATES];
    double center[6];
    double De[6][6];          // per strain component c: sym 3x3
    double* onsite64;
    float* onsite32;
    int* bad;                 // set to 1 on a non-finite input
};

__global__ void onsite_kernel(const FieldArgs a) {
    const long long np = (long long)a.nx * a.ny * a.nz;
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= np) return;
    double v = a.V[p];
    for (int g = 0; g < a.ng; ++g) v += a.alpha[g] * a.levers[(long long)g * np + p];
    double o[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) o[k] = a.center[k] + (k < 3 ? v : 0.0);
    if (a.strain) {
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            const double e = a.strain[(long long)c * np + p];
#pragma unroll
            for (int k = 0; k < 6; ++k) o[k] = fma(a.De[c][k], e, o[k]);
        }
    }
    bool finite = true;
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        finite = finite && isfinite(o[k]);
        a.onsite64[p * 6 + k] = o[k];
        a.onsite32[p * 6 + k] = (float)o[k];
    }
    if (!finite) atomicExch(a.bad, 1);
}

struct PhaseArgs {
    int nx, ny, nz;
    double h;
    double B[3];
    double c[3];      // box centre (symmetric gauge)
    int gauge;
    double2* phase64;
    float2* phase32;
};

__device__ __forceinline__ void vecpot(const PhaseArgs& a, double x, double y, double z, double A[3]) {
    if (a.gauge == 0) {
        const double rx = x - a.c[0], ry = y - a.c[1], rz = z - a.c[2];
        A[0] = 0.5 * (a.B[1] * rz - a.B[2] * ry);
        A[1] = 0.5 * (a.B[2] * rx - a.B[0] * rz);
        A[2] = 0.5 * (a.B[0] * ry - a.B[1] * rx);
    } else {
        A[0] = 0.0;
        A[1] = a.B[2] * x - a.B[0] * z;
        A[2] = -a.B[1] * x;
    }
}

// Peierls phase of the link r -> r' : exp(-i A((r+r')/2).(r'-r) / Phi0).
// Symmetric gauge (mode PH_SYM): A is linear with an antisymmetric gradient,
// so theta(r, r+delta) = A(r).delta / Phi0 = -theta(r, r-delta); only
// (cos, sin) of phi_d = A(r).delta_d / Phi0 is stored per pair.
__global__ void phase_kernel(const PhaseArgs a) {
    const long long np = (long long)a.nx * a.ny * a.nz;
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= np) return;
    const int ix = (int)(p % a.nx);
    const int iy = (int)((p / a.nx) % a.ny);
    const int iz = (int)(p / ((long long)a.nx * a.ny));
    const double x = (ix + 1) * a.h, y = (iy + 1) * a.h, z = (iz + 1) * a.h;
    for (int d = 0; d < 9; ++d) {
        if (a.gauge == 0) {
            const double dx = pair_dx(d) * a.h, dy = pair_dy(d) * a.h, dz = pair_dz(d) * a.h;
            double A[3];
            vecpot(a, x, y, z, A);
            const double phi = (A[0] * dx + A[1] * dy + A[2] * dz) / KHP_PHI0;
            double sn, cs;
            sincos(phi, &sn, &cs);
            a.phase64[p * 9 + d] = make_double2(cs, sn);
            a.phase32[p * 9 + d] = make_float2((float)cs, (float)sn);
            continue;
        }
        for (int sgn = 0; sgn < 2; ++sgn) {
            const double s = sgn == 0 ? 1.0 : -1.0;
            const double dx = s * pair_dx(d) * a.h, dy = s * pair_dy(d) * a.h, dz = s * pair_dz(d) * a.h;
            double A[3];
            vecpot(a, x + 0.5 * dx, y + 0.5 * dy, z + 0.5 * dz, A);
            const double theta = (A[0] * dx + A[1] * dy + A[2] * dz) / KHP_PHI0;
            double sn, cs;
            sincos(theta, &sn, &cs);
            a.phase64[p * 18 + 2 * d + sgn] = make_double2(cs, -sn);
            a.phase32[p * 18 + 2 * d + sgn] = make_float2((float)cs, (float)-sn);
        }
    }
}

cudaError_t launch_field_setup(khp_grid* g, const double* V, const double* strain,
                               const double* levers, const double* alpha, int ng, int* bad) {
    FieldArgs a;
    a.nx = g->nx; a.ny = g->ny; a.nz = g->nz;
    a.V = V; a.strain = strain; a.levers = levers; a.ng = ng;
    for (int i = 0; i < KHP_MAX_GATES; ++i) a.alpha[i] = i < ng ? alpha[i] : 0.0;
    for (int k = 0; k < 6; ++k) a.center[k] = g->center[k];
    for (int c = 0; c < 6; ++c)
        for (int k = 0; k < 6; ++k) a.De[c][k] = g->De[c][k];
    a.onsite64 = g->onsite64; a.onsite32 = g->onsite32; a.bad = bad;
    const int threads = 256;
    const long long blocks = (g->np + threads - 1) / threads;
    onsite_kernel<<<(unsigned)blocks, threads, 0, g->stream>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_phase_setup(g);
}

// Peierls phase tables of the handle's field and gauge; the symmetric gauge
// is taken about the box centre, or about g->ctr when g->ctr_set (a coarse
// grid whose walls sit half a fine step away keeps the fine grid's centre)
cudaError_t launch_phase_setup(khp_grid* g) {
    if (!g->has_phase) return cudaSuccess;
    const int threads = 256;
    const long long blocks = (g->np + threads - 1) / threads;
    PhaseArgs pa;
    pa.nx = g->nx; pa.ny = g->ny; pa.nz = g->nz; pa.h = g->h;
    for (int k = 0; k < 3; ++k) pa.B[k] = g->B[k];
    pa.c[0] = g->ctr_set ? g->ctr[0] : 0.5 * (g->nx + 1) * g->h;
    pa.c[1] = g->ctr_set ? g->ctr[1] : 0.5 * (g->ny + 1) * g->h;
    pa.c[2] = g->ctr_set ? g->ctr[2] : 0.5 * (g->nz + 1) * g->h;
    pa.gauge = g->gauge;
    pa.phase64 = g->phase64; pa.phase32 = g->phase32;
    phase_kernel<<<(unsigned)blocks, threads, 0, g->stream>>>(pa);
    return cudaGetLastError();
}

// --------------------------------------------------- Gershgorin upper bound
// Per point: max over orbital rows of sum_j |onsite_ij| (the rest of the
// Gershgorin row sum is constant and added on the host side of the call).
__global__ void onsite_rowmax_kernel(const double* onsite, long long np, const uint8_t* mask,
                                     double* partial) {
    __shared__ double red[256];
    double m = 0.0;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < np;
         p += (long long)gridDim.x * blockDim.x) {
        if (mask && mask[p] == 0) continue;
        const double* o = onsite + p * 6;
        const double r0 = fabs(o[0]) + fabs(o[5]) + fabs(o[4]);
        const double r1 = fabs(o[5]) + fabs(o[1]) + fabs(o[3]);
        const double r2 = fabs(o[4]) + fabs(o[3]) + fabs(o[2]);
        m = fmax(m, fmax(r0, fmax(r1, r2)));
    }
    red[threadIdx.x] = m;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + s]);
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

__global__ void max_reduce_kernel(const double* partial, int n, double* out) {
    __shared__ double red[256];
    double m = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) m = fmax(m, partial[i]);
    red[threadIdx.x] = m;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + s]);
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = red[0];
}

cudaError_t launch_onsite_rowmax(khp_grid* g, double* partial, int nblocks, double* out) {
    onsite_rowmax_kernel<<<nblocks, 256, 0, g->stream>>>(g->onsite64, g->np, g->mask, partial);
    max_reduce_kernel<<<1, 256, 0, g->stream>>>(partial, nblocks, out);
    return cudaGetLastError();
}

}  // namespace khp
