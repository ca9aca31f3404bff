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
    if ((a.ncol % 2) == 0 && (a.col0 % 2) == 0 && (a.ld % 2) == 0) return launch_vg<R, 2>(a, st);
    return launch_vg<R, 1>(a, st);
}

template cudaError_t launch_stencil<double>(const StencilArgs<double>&, cudaStream_t);
template cudaError_t launch_stencil<float>(const StencilArgs<float>&, cudaStream_t);

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
    if (e != cudaSuccess || !g->has_phase) return e;
    PhaseArgs pa;
    pa.nx = g->nx; pa.ny = g->ny; pa.nz = g->nz; pa.h = g->h;
    for (int k = 0; k < 3; ++k) pa.B[k] = g->B[k];
    pa.c[0] = 0.5 * (g->nx + 1) * g->h;
    pa.c[1] = 0.5 * (g->ny + 1) * g->h;
    pa.c[2] = 0.5 * (g->nz + 1) * g->h;
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
