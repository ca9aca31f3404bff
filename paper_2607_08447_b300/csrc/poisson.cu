// Poisson step of the Schroedinger-Poisson loop (Sec. II B): the potential
// phi (V) of the hole density rho (nm^-3) on the Schroedinger grid, fixed at
// the gate points and with zero normal flux at the box faces elsewhere:
//     sum_{n in nb(p)} (phi_p - phi_n) / h^2 = (e / eps) rho_p      (p not a gate)
//     phi_p = phi_gate(p)                                           (gate)
// nb(p) = face neighbours inside the box.  The gate values move to the
// right-hand side; the remaining operator on the free points is symmetric
// positive definite (some gate in every connected part) and is solved by
// preconditioned conjugate gradients, matrix-free (7-point stencil), every
// scalar on the device; the preconditioner is a geometric multigrid V-cycle
// (default) or the diagonal (Jacobi).  The residual is read back every 8
// (multigrid) or 16 (Jacobi) iterations, the iterations between two reads
// replayed as one captured CUDA graph.  Reductions run in two fixed-order
// stages (deterministic).
#include <algorithm>
#include <cfloat>
#include <cmath>
#include <cstring>
#include <string>
#include <utility>
#include <vector>

#include "khp_common.cuh"
#include "khp_internal.h"

struct khp_poisson_s {
    int nx, ny, nz;
    long long np;
    double h, eps_r, coef, h2inv;
    cudaStream_t stream;
    uint8_t* gate;
    uint16_t* code;        // neighbour codes of the grid's points (see Geo)
    double* gphi;
    int nblk;              // blocks of the kernels with block partials (2 per SM: each thread
                           // takes several points, so the block reductions stay cheap)
    int sblk;              // blocks of the streaming multigrid kernels (8 per SM)
    cudaStream_t work;     // private stream: the CG chunks are captured and replayed on it
    // Anderson mixing of the SP loop (allocated on first use)
    double *a_dv, *a_df;   // [kMaxDepth][np] rings of iterate / residual differences
    double *a_vprev, *a_fprev, *a_f;   // [np]
    double* a_partial;     // [nblk][kMaxR] per-block triangular factors
    double* a_host;        // [nblk][kMaxR] pinned copy of a_partial
    int a_depth, a_count;
    // relaxed-occupation step (allocated on first use)
    double* r_Q;           // [r_nmax][np] potentials of unit occupations (grounded gates)
    double* r_phig;        // [np] potential of the gates alone
    double* r_zero;        // [np] zeros
    double* r_partial;     // block partials of the K and e0 sums
    double* r_out;         // [n][nch][17] sums
    double* r_host;        // pinned copy of r_out
    int r_nmax, r_nq;      // capacity; states whose Q holds a previous solution
    bool r_have_phig;
    // multigrid preconditioner of the CG (FP32): level 0 is the grid itself
    // (its right-hand side is the FP32 copy of the CG residual r; its last
    // sweep writes the CG's z in FP64), levels 1.. the 2x2x2-aggregated grids
    struct MGLevel {
        int nx, ny, nz;
        long long np;
        double h2inv;
        uint8_t* gate;     // level 0: the handle's gate mask
        uint16_t* code;    // level 0: the handle's codes
    };
    static constexpr int kMaxLevels = 12;
    static constexpr int kMaxRhs = 32;
    int mg_n;              // levels; 0 when the hierarchy could not be built
    MGLevel mg[kMaxLevels];
    // the vectors of a CG run over up to cap right-hand sides: [cap][np]
    // (the FP32 multigrid vectors [cap][np_l]), scalars [cap][8] (0 rz,
    // 1 pAp, 2 alpha, 3 beta, 4 rr, 5 bb, 6 max change), block partials
    // [cap][nblk][2]
    struct CGSpace {
        int cap;
        double *x, *r, *z, *p, *Ap, *b, *partial, *s;
        double* host;                      // pinned [cap][8]
        float* mb[kMaxLevels];             // level right-hand sides (level 0: r in FP32)
        float* mu[kMaxLevels];             // smoothing scratch
        float* mv[kMaxLevels];             // level results
        cudaGraphExec_t chunk;             // the iterations between two residual checks
        bool have_chunk;
        int chunk_n;                       // right-hand sides the chunk was captured for
    };
    CGSpace one;           // one right-hand side (its partials and scalars also serve the SP updates)
    CGSpace many;          // up to kMaxRhs right-hand sides, allocated on first use
    float* mg_cinv;        // inverse of the coarsest operator on its free points [nf][nf]
    int* mg_cidx;          // coarsest cell -> free index, -1 at gates
    int mg_nf;
    int precond;           // KHP_POISSON_PRECOND_*
};

namespace khp {
namespace poisson {

constexpr int kT = 256;

__device__ __forceinline__ void coords(long long p, int nx, int ny, int& ix, int& iy, int& iz) {
    ix = (int)(p % nx);
    const long long q = p / nx;
    iy = (int)(q % ny);
    iz = (int)(q / ny);
}

struct Geo {
    int nx, ny, nz;
    long long np;
    double h2inv;
    const uint8_t* gate;
    const uint16_t* code;   // per point: kCodeGate, the degree << 8, bit d = neighbour d in the box and free
    float h2f, h2invf;      // h^2 and h^-2 in FP32 (the multigrid levels)
};

constexpr unsigned kCodeGate = 0x8000u;

__device__ __forceinline__ int code_degree(unsigned c) { return (int)((c >> 8) & 7u); }

// offset of neighbour d (0..5: +x, -x, +y, -y, +z, -z)
__device__ __forceinline__ long long nbr_offset(const Geo& g, int d) {
    const long long sx = 1, sy = g.nx, sz = (long long)g.nx * g.ny;
    return d == 0 ? sx : d == 1 ? -sx : d == 2 ? sy : d == 3 ? -sy : d == 4 ? sz : -sz;
}

// coordinates by 32-bit division (np <= 2^31)
__device__ __forceinline__ void coords32(long long p, int nx, int ny, int& ix, int& iy, int& iz) {
    const unsigned u = (unsigned)p, q = u / (unsigned)nx;
    ix = (int)(u - q * (unsigned)nx);
    iy = (int)(q % (unsigned)ny);
    iz = (int)(q / (unsigned)ny);
}

// neighbour d of p (0..5: +x, -x, +y, -y, +z, -z) or -1 outside the box
__device__ __forceinline__ long long nbr(const Geo& g, long long p, int ix, int iy, int iz, int d) {
    switch (d) {
        case 0: return ix + 1 < g.nx ? p + 1 : -1;
        case 1: return ix > 0 ? p - 1 : -1;
        case 2: return iy + 1 < g.ny ? p + g.nx : -1;
        case 3: return iy > 0 ? p - g.nx : -1;
        case 4: return iz + 1 < g.nz ? p + (long long)g.nx * g.ny : -1;
        default: return iz > 0 ? p - (long long)g.nx * g.ny : -1;
    }
}

// block-partial sums of (a . b) and (c . d) into partial[block][0..1]:
// warp shuffles, then the warps' sums in order (every thread of the block
// calls it)
__device__ __forceinline__ void block_sum2(double va, double vb, double* partial) {
    __shared__ double sa[kT / 32], sb[kT / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        va += __shfl_down_sync(0xffffffffu, va, o);
        vb += __shfl_down_sync(0xffffffffu, vb, o);
    }
    if ((threadIdx.x & 31) == 0) {
        sa[threadIdx.x >> 5] = va;
        sb[threadIdx.x >> 5] = vb;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
#pragma unroll
        for (int w = 0; w < kT / 32; ++w) {
            a += sa[w];
            b += sb[w];
        }
        partial[2 * blockIdx.x] = a;
        partial[2 * blockIdx.x + 1] = b;
    }
}

// Every CG and multigrid kernel runs the right-hand side blockIdx.y of a
// batch: its vectors follow each other at the stride of their level's
// point count (rho and phi at the caller's strides), its scalars at a
// stride of 8, its block partials at a stride of 2 x the launch's blocks.

// b = (e/eps) rho + h^-2 sum_{gate nbrs} phi_gate at free points, 0 at gates;
// x = initial guess at free points, 0 at gates; partial: (b.b, 0)
__global__ void rhs_kernel(const Geo g, const double* rho, long long ld_rho, const double* gphi, double coef,
                           const double* phi_in, long long ld_phi, double* b, double* x, double* partial) {
    const long long k = blockIdx.y;
    rho += k * ld_rho;
    if (phi_in) phi_in += k * ld_phi;
    b += k * g.np;
    x += k * g.np;
    partial += 2 * gridDim.x * k;
    double bb = 0.0;
    for (long long p = (long long)blockIdx.x * kT + threadIdx.x; p < g.np; p += (long long)gridDim.x * kT) {
        if (g.gate[p]) {
            b[p] = 0.0;
            x[p] = 0.0;
            continue;
        }
        int ix, iy, iz;
        coords(p, g.nx, g.ny, ix, iy, iz);
        double v = coef * rho[p];
        for (int d = 0; d < 6; ++d) {
            const long long q = nbr(g, p, ix, iy, iz, d);
            if (q >= 0 && g.gate[q]) v += g.h2inv * gphi[q];
        }
        b[p] = v;
        x[p] = phi_in ? phi_in[p] : 0.0;
        bb += v * v;
    }
    block_sum2(bb, 0.0, partial);
}

// y = A x on free points (0 at gates); partial: (x.y, 0)
__global__ void apply_kernel(const Geo g, const double* __restrict__ x, double* __restrict__ y, double* partial) {
    const long long k = blockIdx.y;
    x += k * g.np;
    y += k * g.np;
    partial += 2 * gridDim.x * k;
    double xy = 0.0;
    for (long long p = (long long)blockIdx.x * kT + threadIdx.x; p < g.np; p += (long long)gridDim.x * kT) {
        const unsigned c = g.code[p];
        if (c & kCodeGate) {
            y[p] = 0.0;
            continue;
        }
        double s = 0.0;
#pragma unroll
        for (int d = 0; d < 6; ++d)
            if (c >> d & 1u) s += x[p + nbr_offset(g, d)];
        const double v = g.h2inv * (code_degree(c) * x[p] - s);
        y[p] = v;
        xy += x[p] * v;
    }
    block_sum2(xy, 0.0, partial);
}

// r = b - A x (A x in y), z = r / diag, p = z; partial: (r.z, r.r)
__global__ void init_kernel(const Geo g, const double* b, const double* Ax, double* r, double* z, double* pv,
                            double* partial) {
    const long long k = blockIdx.y;
    b += k * g.np;
    Ax += k * g.np;
    r += k * g.np;
    z += k * g.np;
    pv += k * g.np;
    partial += 2 * gridDim.x * k;
    double rz = 0.0, rr = 0.0;
    for (long long p = (long long)blockIdx.x * kT + threadIdx.x; p < g.np; p += (long long)gridDim.x * kT) {
        if (g.gate[p]) {
            r[p] = z[p] = pv[p] = 0.0;
            continue;
        }
        int ix, iy, iz;
        coords(p, g.nx, g.ny, ix, iy, iz);
        int deg = 0;
        for (int d = 0; d < 6; ++d) deg += nbr(g, p, ix, iy, iz, d) >= 0;
        const double rv = b[p] - Ax[p];
        const double zv = rv / (g.h2inv * (deg > 0 ? deg : 1));
        r[p] = rv;
        z[p] = zv;
        pv[p] = zv;
        rz += rv * zv;
        rr += rv * rv;
    }
    block_sum2(rz, rr, partial);
}

// x += alpha p, r -= alpha Ap, z = r / diag; partial: (r.z, r.r)
__global__ void update_kernel(const Geo g, const double* s, const double* pv, const double* Ap, double* x, double* r,
                              double* z, double* partial) {
    const long long k = blockIdx.y;
    pv += k * g.np;
    Ap += k * g.np;
    x += k * g.np;
    r += k * g.np;
    z += k * g.np;
    partial += 2 * gridDim.x * k;
    const double alpha = s[8 * k + 2];
    double rz = 0.0, rr = 0.0;
    for (long long p = (long long)blockIdx.x * kT + threadIdx.x; p < g.np; p += (long long)gridDim.x * kT) {
        const unsigned c = g.code[p];
        if (c & kCodeGate) continue;
        const int deg = code_degree(c);
        x[p] += alpha * pv[p];
        const double rv = r[p] - alpha * Ap[p];
        const double zv = rv / (g.h2inv * (deg > 0 ? deg : 1));
        r[p] = rv;
        z[p] = zv;
        rz += rv * zv;
        rr += rv * rv;
    }
    block_sum2(rz, rr, partial);
}

// p = z + beta p
__global__ void direction_kernel(const Geo g, const double* s, const double* z, double* pv) {
    const long long k = blockIdx.y;
    z += k * g.np;
    pv += k * g.np;
    const double beta = s[8 * k + 3];
    for (long long p = (long long)blockIdx.x * kT + threadIdx.x; p < g.np; p += (long long)gridDim.x * kT)
        if (!g.gate[p]) pv[p] = z[p] + beta * pv[p];
}

// ------------------------------------------------- multigrid preconditioner
// Cell-centred geometric multigrid V-cycle on the Poisson operator, in
// FP32 (a preconditioner needs no more: the CG's residual, iterate and dot
// products stay FP64, and FP32 arithmetic runs at many times B300's FP64
// rate).  Level l+1 aggregates 2x2x2 cells of level l (the last cell along
// an odd dimension has one child along it); its spacing doubles and a
// coarse cell is a gate when any of its children is.  The coarse operator
// is the same 7-point form rediscretised at the coarse spacing with zero
// gate values (the levels solve for corrections).  Restriction averages
// the 8 children, prolongation adds the coarse value to every free child,
// two weighted-Jacobi sweeps (omega = 0.8) run before and after the coarse
// correction, and the coarsest level (at most 64 cells) is solved by a
// dense inverse.  Restriction is 1/8 of the transposed prolongation and
// the smoothing is symmetric, so the V-cycle is a symmetric preconditioner
// for the CG.  The rediscretised coarse operator is half the Galerkin one
// (R A P), so the coarse correction is twice the A-orthogonal projection:
// the usual remedy for the too-small correction that piecewise-constant
// prolongation gives on smooth errors.
//
// A Jacobi sweep y -> y + w D^-1 (b - A y), D = deg / h^2, is evaluated as
// (1 - w) y + (w / deg) (sum of the free neighbours' y + h^2 b).
constexpr float kOmega = 0.8f;

__device__ __forceinline__ long long idx_of(const Geo& g, int ix, int iy, int iz) {
    return ix + (long long)g.nx * (iy + (long long)g.ny * iz);
}

// 1 / max(deg, 1) of a point's code
__device__ __forceinline__ float inv_deg(unsigned c) {
    const int d = code_degree(c);
    return d == 6 ? 1.0f / 6.0f : d == 5 ? 0.2f : d == 4 ? 0.25f : d == 3 ? 1.0f / 3.0f : d == 2 ? 0.5f : 1.0f;
}

// the neighbour code of every point of a level (from its gate mask)
__global__ void mg_code_kernel(const Geo g, uint16_t* code) {
    for (long long p = (long long)blockIdx.x * kT + threadIdx.x; p < g.np; p += (long long)gridDim.x * kT) {
        int ix, iy, iz;
        coords32(p, g.nx, g.ny, ix, iy, iz);
        const bool in[6] = {ix + 1 < g.nx, ix > 0, iy + 1 < g.ny, iy > 0, iz + 1 < g.nz, iz > 0};
        unsigned c = g.gate[p] ? kCodeGate : 0u;
        int deg = 0;
        for (int d = 0; d < 6; ++d) {
            if (!in[d]) continue;
            ++deg;
            if (!g.gate[p + nbr_offset(g, d)]) c |= 1u << d;
        }
        code[p] = (uint16_t)(c | (unsigned)deg << 8);
    }
}

// pre-smoothing from a zero start, both sweeps in one pass:
// u = w D^-1 b, v = u + w D^-1 (b - A u) (u of the neighbours recomputed); 0 at gates
__global__ void mg_presmooth_kernel(const Geo g, const float* __restrict__ b, float* __restrict__ v) {
    b += blockIdx.y * g.np;
    v += blockIdx.y * g.np;
    const float wh2 = kOmega * g.h2f;
    for (long long p = (long long)blockIdx.x * kT + threadIdx.x; p < g.np; p += (long long)gridDim.x * kT) {
        const unsigned c = g.code[p];
        if (c & kCodeGate) {
            v[p] = 0.0f;
            continue;
        }
        float s = 0.0f;
#pragma unroll
        for (int d = 0; d < 6; ++d)
            if (c >> d & 1u) {
                const long long q = p + nbr_offset(g, d);
                s = fmaf(b[q], inv_deg(g.code[q]), s);
            }
        const float id = inv_deg(c), bp = b[p];
        const float up = wh2 * bp * id;
        v[p] = fmaf(1.0f - kOmega, up, kOmega * id * fmaf(g.h2f, bp, wh2 * s));
    }
}

// coarse right-hand side: the mean of the residuals b - A v of the 8
// children (a free coarse cell has only free children); 0 at coarse gates.
// Eight consecutive lanes per coarse cell, one child each, summed by
// shuffles in a fixed order.
__global__ void mg_restrict_kernel(const Geo f, const float* __restrict__ v, const float* __restrict__ b,
                                   const Geo c, float* __restrict__ bc) {
    v += blockIdx.y * f.np;
    b += blockIdx.y * f.np;
    bc += blockIdx.y * c.np;
    const long long n8 = 8 * c.np;
    // n8 and the stride are multiples of 8: the 8 lanes of a cell run every iteration together
    for (long long t = (long long)blockIdx.x * kT + threadIdx.x; t < n8; t += (long long)gridDim.x * kT) {
        const long long q = t >> 3;
        const int k = (int)(t & 7);
        const bool cgate = (c.code[q] & kCodeGate) != 0;
        float res = 0.0f;
        if (!cgate) {
            int jx, jy, jz;
            coords32(q, c.nx, c.ny, jx, jy, jz);
            const int ix = 2 * jx + (k & 1), iy = 2 * jy + ((k >> 1) & 1), iz = 2 * jz + (k >> 2);
            if (ix < f.nx && iy < f.ny && iz < f.nz) {
                const long long p = idx_of(f, ix, iy, iz);
                const unsigned cp = f.code[p];
                if (!(cp & kCodeGate)) {
                    float sn = 0.0f;
#pragma unroll
                    for (int d = 0; d < 6; ++d)
                        if (cp >> d & 1u) sn += v[p + nbr_offset(f, d)];
                    res = b[p] - f.h2invf * fmaf((float)code_degree(cp), v[p], -sn);
                }
            }
        }
        const unsigned mask = 0xFFu << (threadIdx.x & 24u);
        res += __shfl_xor_sync(mask, res, 1);
        res += __shfl_xor_sync(mask, res, 2);
        res += __shfl_xor_sync(mask, res, 4);
        if (k == 0) bc[q] = cgate ? 0.0f : 0.125f * res;
    }
}

// coarsest level: x = A^-1 b on its free points (one CTA, dense inverse of at most 64 x 64)
__global__ void __launch_bounds__(kT) mg_coarse_kernel(const Geo c, const float* __restrict__ b,
                                                       float* __restrict__ x, const float* __restrict__ cinv,
                                                       const int* __restrict__ cidx, int nf) {
    b += blockIdx.x * c.np;     // one CTA per right-hand side
    x += blockIdx.x * c.np;
    __shared__ float bf[64];
    for (int p = threadIdx.x; p < (int)c.np; p += kT)
        if (cidx[p] >= 0) bf[cidx[p]] = b[p];
    __syncthreads();
    for (int p = threadIdx.x; p < (int)c.np; p += kT) {
        const int i = cidx[p];
        float s = 0.0f;
        if (i >= 0)
            for (int j = 0; j < nf; ++j) s = fmaf(cinv[i * nf + j], bf[j], s);
        x[p] = s;
    }
}

// one weighted-Jacobi sweep xout = y + w D^-1 (b - A y) with y = xin, plus
// with kCoarse the coarse correction xc of the parent cell (the
// prolongation fused into the first post-smoothing sweep); 0 at gates.
// kLast (the last sweep on the grid itself): the result goes to z in FP64,
// with the block sums of (r.z, r.r) over the FP64 residual r into partial.
template <bool kCoarse, bool kLast>
__global__ void mg_smooth_kernel(const Geo g, const float* __restrict__ xin, const Geo c,
                                 const float* __restrict__ xc, const float* __restrict__ b,
                                 float* __restrict__ xout, const double* __restrict__ r, double* __restrict__ z,
                                 double* partial) {
    const long long k = blockIdx.y;
    xin += k * g.np;
    b += k * g.np;
    if constexpr (kCoarse) xc += k * c.np;
    if constexpr (kLast) {
        r += k * g.np;
        z += k * g.np;
        partial += 2 * gridDim.x * k;
    } else {
        xout += k * g.np;
    }
    double rz = 0.0, rr = 0.0;
    for (long long p = (long long)blockIdx.x * kT + threadIdx.x; p < g.np; p += (long long)gridDim.x * kT) {
        const unsigned cp = g.code[p];
        if (cp & kCodeGate) {
            if constexpr (kLast) z[p] = 0.0;
            else xout[p] = 0.0f;
            continue;
        }
        float yp = xin[p], s = 0.0f;
        if constexpr (kCoarse) {
            int ix, iy, iz;
            coords32(p, g.nx, g.ny, ix, iy, iz);
            yp += xc[idx_of(c, ix >> 1, iy >> 1, iz >> 1)];
#pragma unroll
            for (int d = 0; d < 6; ++d)
                if (cp >> d & 1u) {
                    const int qx = ix + (d == 0) - (d == 1), qy = iy + (d == 2) - (d == 3), qz = iz + (d == 4) - (d == 5);
                    s += xin[p + nbr_offset(g, d)] + xc[idx_of(c, qx >> 1, qy >> 1, qz >> 1)];
                }
        } else {
#pragma unroll
            for (int d = 0; d < 6; ++d)
                if (cp >> d & 1u) s += xin[p + nbr_offset(g, d)];
        }
        const float out = fmaf(1.0f - kOmega, yp, kOmega * inv_deg(cp) * fmaf(g.h2f, b[p], s));
        if constexpr (kLast) {
            const double zd = (double)out, rd = r[p];
            z[p] = zd;
            rz = fma(rd, zd, rz);
            rr = fma(rd, rd, rr);
        } else {
            xout[p] = out;
        }
    }
    if constexpr (kLast) block_sum2(rz, rr, partial);
}

// z = x (FP32 result of a V-cycle that is the coarsest solve alone) in FP64; partial: (r.z, r.r)
__global__ void mg_out_kernel(const Geo g, const float* x, const double* r, double* z, double* partial) {
    const long long k = blockIdx.y;
    x += k * g.np;
    r += k * g.np;
    z += k * g.np;
    partial += 2 * gridDim.x * k;
    double rz = 0.0, rr = 0.0;
    for (long long p = (long long)blockIdx.x * kT + threadIdx.x; p < g.np; p += (long long)gridDim.x * kT) {
        const double zd = g.gate[p] ? 0.0 : (double)x[p], rd = r[p];
        z[p] = zd;
        rz = fma(rd, zd, rz);
        rr = fma(rd, rd, rr);
    }
    block_sum2(rz, rr, partial);
}

// CG steps around the multigrid preconditioner:
// r = b - A x (A x in Ax) and its FP32 copy rf, 0 at gates
__global__ void init_mg_kernel(const Geo g, const double* b, const double* Ax, double* r, float* rf) {
    const long long k = blockIdx.y;
    b += k * g.np;
    Ax += k * g.np;
    r += k * g.np;
    rf += k * g.np;
    for (long long p = (long long)blockIdx.x * kT + threadIdx.x; p < g.np; p += (long long)gridDim.x * kT) {
        const double v = g.gate[p] ? 0.0 : b[p] - Ax[p];
        r[p] = v;
        rf[p] = (float)v;
    }
}

// x += alpha p, r -= alpha Ap, rf = r in FP32
__global__ void update_mg_kernel(const Geo g, const double* s, const double* pv, const double* Ap, double* x,
                                 double* r, float* rf) {
    const long long k = blockIdx.y;
    pv += k * g.np;
    Ap += k * g.np;
    x += k * g.np;
    r += k * g.np;
    rf += k * g.np;
    const double alpha = s[8 * k + 2];
    for (long long p = (long long)blockIdx.x * kT + threadIdx.x; p < g.np; p += (long long)gridDim.x * kT) {
        if (g.code[p] & kCodeGate) continue;
        x[p] += alpha * pv[p];
        const double v = r[p] - alpha * Ap[p];
        r[p] = v;
        rf[p] = (float)v;
    }
}

// coarse gate mask: a coarse cell is a gate when any child is
__global__ void mg_gate_kernel(const Geo f, const Geo c, uint8_t* gc) {
    for (long long q = (long long)blockIdx.x * kT + threadIdx.x; q < c.np; q += (long long)gridDim.x * kT) {
        int jx, jy, jz;
        coords(q, c.nx, c.ny, jx, jy, jz);
        uint8_t gv = 0;
        for (int k = 0; k < 8; ++k) {
            const int ix = 2 * jx + (k & 1), iy = 2 * jy + ((k >> 1) & 1), iz = 2 * jz + (k >> 2);
            if (ix < f.nx && iy < f.ny && iz < f.nz && f.gate[idx_of(f, ix, iy, iz)]) gv = 1;
        }
        gc[q] = gv;
    }
}

// one block sums the block partials (thread t takes partials t, t + 256, ...
// in order, then a fixed tree), so the result does not depend on timing;
// mode selects the update
//  0: s[5] = bb                      (after rhs_kernel)
//  1: s[0] = rz, s[4] = rr           (after init_kernel)
//  2: s[1] = pAp, s[2] = rz / pAp    (after apply_kernel on p)
//  3: s[3] = rz_new / rz, s[0] = rz_new, s[4] = rr   (after update_kernel)
__global__ void __launch_bounds__(kT) finish_kernel(const double* partial, int nblk, int mode, double* s) {
    partial += 2 * (long long)nblk * blockIdx.x;   // one CTA per right-hand side
    s += 8 * blockIdx.x;
    __shared__ double sa[kT], sb[kT];
    double a = 0.0, b = 0.0;
    for (int k = threadIdx.x; k < nblk; k += kT) {
        a += partial[2 * k];
        b += partial[2 * k + 1];
    }
    sa[threadIdx.x] = a;
    sb[threadIdx.x] = b;
    __syncthreads();
    for (int st = kT / 2; st > 0; st >>= 1) {
        if (threadIdx.x < st) {
            sa[threadIdx.x] += sa[threadIdx.x + st];
            sb[threadIdx.x] += sb[threadIdx.x + st];
        }
        __syncthreads();
    }
    if (threadIdx.x != 0) return;
    a = sa[0];
    b = sb[0];
    if (mode == 0) s[5] = a;
    else if (mode == 1) { s[0] = a; s[4] = b; }
    else if (mode == 2) { s[1] = a; s[2] = a != 0.0 ? s[0] / a : 0.0; }
    else { s[3] = s[0] != 0.0 ? a / s[0] : 0.0; s[0] = a; s[4] = b; }
}

// phi = x at free points, phi_gate at gates
__global__ void output_kernel(const Geo g, const double* x, const double* gphi, double* phi, long long ld_phi) {
    x += blockIdx.y * g.np;
    phi += blockIdx.y * ld_phi;
    for (long long p = (long long)blockIdx.x * kT + threadIdx.x; p < g.np; p += (long long)gridDim.x * kT)
        phi[p] = g.gate[p] ? gphi[p] : x[p];
}

// V = (1 - a) V + a (V_ext + phi); partial: (max |dV|, 0)
__global__ void mix_kernel(long long np, const double* Vext, const double* phi, double a, double* V, double* partial) {
    __shared__ double sm[kT];
    double mx = 0.0;
    for (long long p = (long long)blockIdx.x * kT + threadIdx.x; p < np; p += (long long)gridDim.x * kT) {
        const double v = V[p];
        const double vn = (1.0 - a) * v + a * ((Vext ? Vext[p] : 0.0) + phi[p]);
        V[p] = vn;
        mx = fmax(mx, fabs(vn - v));
    }
    sm[threadIdx.x] = mx;
    __syncthreads();
    for (int st = kT / 2; st > 0; st >>= 1) {
        if (threadIdx.x < st) sm[threadIdx.x] = fmax(sm[threadIdx.x], sm[threadIdx.x + st]);
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[2 * blockIdx.x] = sm[0];
}

__global__ void __launch_bounds__(kT) max_finish_kernel(const double* partial, int nblk, double* out) {
    __shared__ double sm[kT];
    double m = 0.0;
    for (int k = threadIdx.x; k < nblk; k += kT) m = fmax(m, partial[2 * k]);
    sm[threadIdx.x] = m;
    __syncthreads();
    for (int st = kT / 2; st > 0; st >>= 1) {
        if (threadIdx.x < st) sm[threadIdx.x] = fmax(sm[threadIdx.x], sm[threadIdx.x + st]);
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sm[0];
}

// ------------------------------------------------------------------------
// Anderson mixing (type II) for the fixed point V = G(V) = V_ext + phi[V]:
// F_k = G(V_k) - V_k; history columns dV_i = V_{i+1} - V_i and
// dF_i = F_{i+1} - F_i of the last m steps; gamma = argmin |F_k - dF gamma|;
// V_{k+1} = V_k + beta F_k - sum_i gamma_i (dV_i + beta dF_i).
// The least squares is solved through a QR factorisation of the tall
// matrix A = [dF | F] (Np x (m+1)) without forming A^T A: every thread
// folds its rows into a triangular factor by Givens rotations, the factors
// of a block are merged the same way (a tall-skinny QR), and the host
// merges the blocks' factors and solves R11 gamma = r12 through the SVD of
// R11 (least-squares semantics for a rank-deficient history).
constexpr int kMaxDepth = 8;
constexpr int kMaxR = (kMaxDepth + 1) * (kMaxDepth + 2) / 2;   // packed (m+1)x(m+1) upper triangle

__global__ void anderson_residual_kernel(long long np, const double* Vext, const double* phi, const double* V,
                                         double* f, double* vprev, double* fprev, double* dv, double* df) {
    for (long long p = (long long)blockIdx.x * kT + threadIdx.x; p < np; p += (long long)gridDim.x * kT) {
        const double v = V[p];
        const double F = (Vext ? Vext[p] : 0.0) + phi[p] - v;
        f[p] = F;
        if (dv) {
            dv[p] = v - vprev[p];
            df[p] = F - fprev[p];
        }
        vprev[p] = v;
        fprev[p] = F;
    }
}

// Packed row-major upper triangle of a C x C matrix: row k holds columns
// k..C-1 starting at offset k C - k (k - 1) / 2.
__host__ __device__ constexpr int tri_at(int C, int k) { return k * C - k * (k - 1) / 2; }

// Fold the row a (C entries) into the triangular factor R by Givens
// rotations, so that R^T R gains a a^T.
template <int C>
__device__ __forceinline__ void givens_fold(double (&R)[C * (C + 1) / 2], double (&a)[C]) {
#pragma unroll
    for (int k = 0; k < C; ++k) {
        const int rk = tri_at(C, k);
        const double y = a[k];
        if (y != 0.0) {
            const double x = R[rk];
            const double r = hypot(x, y);
            const double c = x / r, sn = y / r;
            R[rk] = r;
#pragma unroll
            for (int j = k + 1; j < C; ++j) {
                const double rj = R[rk + j - k];
                R[rk + j - k] = c * rj + sn * a[j];
                a[j] = c * a[j] - sn * rj;
            }
        }
    }
}

// Fold every row of another factor Q into R.
template <int C>
__device__ __forceinline__ void givens_merge(double (&R)[C * (C + 1) / 2], const double (&Q)[C * (C + 1) / 2]) {
#pragma unroll
    for (int k = 0; k < C; ++k) {
        double a[C];
#pragma unroll
        for (int j = 0; j < C; ++j) a[j] = j < k ? 0.0 : Q[tri_at(C, k) + j - k];
        givens_fold<C>(R, a);
    }
}

// One triangular factor of [dF_0 .. dF_{M-1} | F] per block into
// partial[block][C (C + 1) / 2], C = M + 1.
template <int M>
__global__ void __launch_bounds__(kT) anderson_qr_kernel(long long np, const double* __restrict__ df,
                                                         const double* __restrict__ f, double* partial) {
    constexpr int C = M + 1;
    constexpr int K = C * (C + 1) / 2;
    double R[K];
#pragma unroll
    for (int k = 0; k < K; ++k) R[k] = 0.0;
    for (long long p = (long long)blockIdx.x * kT + threadIdx.x; p < np; p += (long long)gridDim.x * kT) {
        double a[C];
#pragma unroll
        for (int i = 0; i < M; ++i) a[i] = df[(long long)i * np + p];
        a[M] = f[p];
        givens_fold<C>(R, a);
    }
    // merge within the warp, halving the active lanes each level
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll 1
    for (int off = 16; off > 0; off >>= 1) {
        double Q[K];
#pragma unroll
        for (int k = 0; k < K; ++k) Q[k] = __shfl_down_sync(0xffffffffu, R[k], off);
        if (lane < off) givens_merge<C>(R, Q);
    }
    __shared__ double sm[kT / 32][K];
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < K; ++k) sm[warp][k] = R[k];
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll 1
        for (int w = 1; w < kT / 32; ++w) {
            double Q[K];
#pragma unroll
            for (int k = 0; k < K; ++k) Q[k] = sm[w][k];
            givens_merge<C>(R, Q);
        }
#pragma unroll
        for (int k = 0; k < K; ++k) partial[(size_t)blockIdx.x * K + k] = R[k];
    }
}

struct AndersonCoef {
    double gamma[kMaxDepth];
};

__global__ void anderson_update_kernel(long long np, int m, double beta, const AndersonCoef c, double* V,
                                       const double* f, const double* dv, const double* df, double* partial) {
    __shared__ double sm[kT];
    double mx = 0.0;
    for (long long p = (long long)blockIdx.x * kT + threadIdx.x; p < np; p += (long long)gridDim.x * kT) {
        const double v = V[p];
        double vn = v + beta * f[p];
        for (int i = 0; i < m; ++i)
            vn -= c.gamma[i] * (dv[(long long)i * np + p] + beta * df[(long long)i * np + p]);
        V[p] = vn;
        mx = fmax(mx, fabs(vn - v));
    }
    sm[threadIdx.x] = mx;
    __syncthreads();
    for (int st = kT / 2; st > 0; st >>= 1) {
        if (threadIdx.x < st) sm[threadIdx.x] = fmax(sm[threadIdx.x], sm[threadIdx.x + st]);
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[2 * blockIdx.x] = sm[0];
}

// ------------------------------------------------------------------------
// Relaxed occupations (Schroedinger-Poisson loop): with the per-state
// densities dens_i, the unit-occupation potentials Q_j and the gate
// potential phi_g, the sums
//     K_ij = sum_p dens_i(p) Q_j(p),
//     d_i  = sum_p dens_i(p) (phi_g(p) - (V(p) - V_ext(p)))
// in fixed order: block partials of 16 j's (plus d_i in chunk 0) per
// (i, chunk), then one block per (i, chunk) over the partials.
constexpr int kRJ = 16;

__global__ void __launch_bounds__(kT) relax_dots_kernel(long long np, int n, const double* __restrict__ dens,
                                                        const double* __restrict__ Q, const double* __restrict__ phig,
                                                        const double* __restrict__ V, const double* __restrict__ Vext,
                                                        double* __restrict__ partial) {
    const int i = blockIdx.y, jc = blockIdx.z, nch = gridDim.z;
    const int j0 = jc * kRJ;
    double acc[kRJ + 1];
#pragma unroll
    for (int k = 0; k <= kRJ; ++k) acc[k] = 0.0;
    const double* di = dens + (long long)i * np;
    for (long long p = (long long)blockIdx.x * kT + threadIdx.x; p < np; p += (long long)gridDim.x * kT) {
        const double w = di[p];
#pragma unroll
        for (int k = 0; k < kRJ; ++k)
            if (j0 + k < n) acc[k] = fma(w, Q[(long long)(j0 + k) * np + p], acc[k]);
        if (jc == 0) acc[kRJ] = fma(w, phig[p] - (V[p] - (Vext ? Vext[p] : 0.0)), acc[kRJ]);
    }
    __shared__ double sm[kT / 32][kRJ + 1];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k <= kRJ; ++k) {
        double v = acc[k];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) sm[warp][k] = v;
    }
    __syncthreads();
    if (threadIdx.x <= kRJ) {
        double v = 0.0;
        for (int w = 0; w < kT / 32; ++w) v += sm[w][threadIdx.x];
        partial[(((long long)i * nch + jc) * gridDim.x + blockIdx.x) * (kRJ + 1) + threadIdx.x] = v;
    }
}

__global__ void relax_sum_kernel(const double* partial, int nblk, double* out) {
    const int row = blockIdx.x, k = threadIdx.x;
    if (k > kRJ) return;
    double v = 0.0;
    for (int b = 0; b < nblk; ++b) v += partial[((long long)row * nblk + b) * (kRJ + 1) + k];
    out[row * (kRJ + 1) + k] = v;
}

struct RelaxCoef {
    double f[KHP_MAX_M];
};

// phi = phi_g + sum_j f_j Q_j
__global__ void relax_combine_kernel(long long np, int n, const RelaxCoef c, const double* __restrict__ phig,
                                     const double* __restrict__ Q, double* __restrict__ phi) {
    for (long long p = (long long)blockIdx.x * kT + threadIdx.x; p < np; p += (long long)gridDim.x * kT) {
        double v = phig[p];
        for (int j = 0; j < n; ++j) v = fma(c.f[j], Q[(long long)j * np + p], v);
        phi[p] = v;
    }
}

__global__ void copy_gate_values_kernel(long long np, const uint8_t* gate, const double* src, double* gphi) {
    for (long long p = (long long)blockIdx.x * kT + threadIdx.x; p < np; p += (long long)gridDim.x * kT)
        gphi[p] = gate[p] ? src[p] : 0.0;
}

}  // namespace poisson
}  // namespace khp

// ------------------------------------------------------------------ C ABI
namespace {

using khp::poisson::kT;

khp_status pfail(khp_status s, const std::string& m) { return khp_set_error(s, m); }

#define CKSP(call)                                                                          \
    do {                                                                                    \
        const khp_status s_ = (call);                                                       \
        if (s_ != KHP_OK) return s_;                                                        \
    } while (0)

// launch check with the step's name in the message
#define PCKL(what)                                                                          \
    do {                                                                                    \
        const cudaError_t e_ = cudaGetLastError();                                          \
        if (e_ != cudaSuccess) return pfail(KHP_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e_)); \
    } while (0)

#define PCK(call)                                                                           \
    do {                                                                                    \
        const cudaError_t e_ = (call);                                                      \
        if (e_ != cudaSuccess) return pfail(KHP_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

khp::poisson::Geo geo(const khp_poisson_s* P) {
    khp::poisson::Geo g;
    g.nx = P->nx; g.ny = P->ny; g.nz = P->nz; g.np = P->np; g.h2inv = P->h2inv; g.gate = P->gate;
    g.code = P->code;
    g.h2f = (float)(1.0 / P->h2inv);
    g.h2invf = (float)P->h2inv;
    return g;
}

khp::poisson::Geo mg_geo(const khp_poisson_s* P, int l) {
    const khp_poisson_s::MGLevel& L = P->mg[l];
    khp::poisson::Geo g;
    g.nx = L.nx; g.ny = L.ny; g.nz = L.nz; g.np = L.np; g.h2inv = L.h2inv; g.gate = L.gate;
    g.code = L.code;
    g.h2f = (float)(1.0 / L.h2inv);
    g.h2invf = (float)L.h2inv;
    return g;
}

void mg_free(khp_poisson_s* P) {
    for (int l = 1; l < khp_poisson_s::kMaxLevels; ++l) {
        khp_poisson_s::MGLevel& L = P->mg[l];
        if (L.gate) cudaFree(L.gate);
        if (L.code) cudaFree(L.code);
    }
    for (auto& L : P->mg) L = khp_poisson_s::MGLevel{};
    if (P->mg_cinv) cudaFree(P->mg_cinv);
    if (P->mg_cidx) cudaFree(P->mg_cidx);
    P->mg_cinv = nullptr;
    P->mg_cidx = nullptr;
    P->mg_n = 0;
}

void space_free(khp_poisson_s::CGSpace& w) {
    if (w.have_chunk) cudaGraphExecDestroy(w.chunk);
    double* bufs[] = {w.x, w.r, w.z, w.p, w.Ap, w.b, w.partial, w.s};
    for (double* b : bufs)
        if (b) cudaFree(b);
    if (w.host) cudaFreeHost(w.host);
    for (int l = 0; l < khp_poisson_s::kMaxLevels; ++l) {
        if (w.mb[l]) cudaFree(w.mb[l]);
        if (w.mu[l]) cudaFree(w.mu[l]);
        if (w.mv[l]) cudaFree(w.mv[l]);
    }
    w = khp_poisson_s::CGSpace{};
}

// the vectors of cap right-hand sides (the multigrid ones for the levels built)
cudaError_t space_alloc(khp_poisson_s* P, khp_poisson_s::CGSpace& w, int cap) {
    space_free(w);
    w.cap = cap;
    const size_t vb = sizeof(double) * (size_t)P->np * cap;
    cudaError_t e;
    if ((e = cudaMalloc(&w.x, vb)) != cudaSuccess || (e = cudaMalloc(&w.r, vb)) != cudaSuccess ||
        (e = cudaMalloc(&w.z, vb)) != cudaSuccess || (e = cudaMalloc(&w.p, vb)) != cudaSuccess ||
        (e = cudaMalloc(&w.Ap, vb)) != cudaSuccess || (e = cudaMalloc(&w.b, vb)) != cudaSuccess ||
        (e = cudaMalloc(&w.partial, sizeof(double) * 2 * P->nblk * cap)) != cudaSuccess ||
        (e = cudaMalloc(&w.s, sizeof(double) * 8 * cap)) != cudaSuccess ||
        (e = cudaMallocHost(&w.host, sizeof(double) * 8 * cap)) != cudaSuccess)
        return e;
    for (int l = 0; l < P->mg_n; ++l) {
        const size_t fb = sizeof(float) * (size_t)P->mg[l].np * cap;
        if ((e = cudaMalloc(&w.mb[l], fb)) != cudaSuccess || (e = cudaMalloc(&w.mu[l], fb)) != cudaSuccess ||
            (e = cudaMalloc(&w.mv[l], fb)) != cudaSuccess)
            return e;
    }
    return cudaSuccess;
}

void free_all(khp_poisson_s* P) {
    space_free(P->one);
    space_free(P->many);
    mg_free(P);
    if (P->work) cudaStreamDestroy(P->work);
    double* bufs[] = {P->gphi, P->a_dv, P->a_df, P->a_vprev, P->a_fprev, P->a_f, P->a_partial,
                      P->r_Q, P->r_phig, P->r_zero, P->r_partial, P->r_out};
    for (double* b : bufs)
        if (b) cudaFree(b);
    if (P->gate) cudaFree(P->gate);
    if (P->code) cudaFree(P->code);
    if (P->a_host) cudaFreeHost(P->a_host);
    if (P->r_host) cudaFreeHost(P->r_host);
}

int mg_blocks(long long np, int nblk) { return (int)std::min<long long>((np + kT - 1) / kT, nblk); }

// Builds the multigrid hierarchy (geometry, gate masks, codes, coarsest
// inverse; the vectors belong to the CG spaces) of the handle's grid and
// gate mask on the handle's stream (synchronous).  Leaves mg_n = 0 (Jacobi preconditioner
// only) when the grid does not coarsen to at most 64 cells within
// kMaxLevels levels, or when the coarsest operator is not positive definite
// (a grid without gates, whose Poisson operator is singular).
khp_status mg_build(khp_poisson_s* P) {
    using namespace khp::poisson;
    using MGLevel = khp_poisson_s::MGLevel;
    constexpr int kMaxL = khp_poisson_s::kMaxLevels;
    int dims[kMaxL][3] = {{P->nx, P->ny, P->nz}};
    auto npl = [&](int l) { return (long long)dims[l][0] * dims[l][1] * dims[l][2]; };
    int L = 1;
    while (npl(L - 1) > 64 && L < kMaxL) {
        for (int a = 0; a < 3; ++a) dims[L][a] = (dims[L - 1][a] + 1) / 2;
        ++L;
    }
    if (npl(L - 1) > 64) return KHP_OK;
    cudaError_t e = cudaSuccess;
    for (int l = 0; l < L && e == cudaSuccess; ++l) {
        MGLevel& M = P->mg[l];
        M.nx = dims[l][0]; M.ny = dims[l][1]; M.nz = dims[l][2];
        M.np = npl(l);
        M.h2inv = std::ldexp(P->h2inv, -2 * l);
        if (l == 0) {
            M.gate = P->gate;
            M.code = P->code;
        } else if ((e = cudaMalloc(&M.gate, M.np)) == cudaSuccess) {
            e = cudaMalloc(&M.code, sizeof(uint16_t) * M.np);
        }
    }
    if (e != cudaSuccess) {
        mg_free(P);
        return pfail(KHP_ERR_OOM, std::string("multigrid levels: ") + cudaGetErrorString(e));
    }
    for (int l = 1; l < L; ++l) {
        const int nb = mg_blocks(P->mg[l].np, P->sblk);
        mg_gate_kernel<<<nb, kT, 0, P->stream>>>(mg_geo(P, l - 1), mg_geo(P, l), P->mg[l].gate);
        mg_code_kernel<<<nb, kT, 0, P->stream>>>(mg_geo(P, l), P->mg[l].code);
    }
    const MGLevel& C = P->mg[L - 1];
    const int nc = (int)C.np;
    std::vector<uint8_t> gh(nc);
    if ((e = cudaGetLastError()) != cudaSuccess ||
        (e = cudaMemcpyAsync(gh.data(), C.gate, nc, cudaMemcpyDeviceToHost, P->stream)) != cudaSuccess ||
        (e = cudaStreamSynchronize(P->stream)) != cudaSuccess) {
        mg_free(P);
        return pfail(KHP_ERR_CUDA, std::string("multigrid gate masks: ") + cudaGetErrorString(e));
    }
    // the coarsest operator on its free cells, the same 7-point rule as the kernels
    std::vector<int> idx(nc, -1);
    int nf = 0;
    for (int q = 0; q < nc; ++q)
        if (!gh[q]) idx[q] = nf++;
    std::vector<double> A((size_t)nf * nf, 0.0);
    std::vector<float> inv((size_t)std::max(nf, 1) * std::max(nf, 1), 0.0f);
    for (int q = 0; q < nc; ++q) {
        if (idx[q] < 0) continue;
        const int ix = q % C.nx, iy = (q / C.nx) % C.ny, iz = q / (C.nx * C.ny);
        const int nb[6][3] = {{ix + 1, iy, iz}, {ix - 1, iy, iz}, {ix, iy + 1, iz},
                              {ix, iy - 1, iz}, {ix, iy, iz + 1}, {ix, iy, iz - 1}};
        int deg = 0;
        for (const auto& n : nb) {
            if (n[0] < 0 || n[0] >= C.nx || n[1] < 0 || n[1] >= C.ny || n[2] < 0 || n[2] >= C.nz) continue;
            ++deg;
            const int j = idx[n[0] + C.nx * (n[1] + C.ny * n[2])];
            if (j >= 0) A[(size_t)idx[q] * nf + j] -= C.h2inv;
        }
        A[(size_t)idx[q] * nf + idx[q]] += C.h2inv * deg;
    }
    // Cholesky A = G G^T (lower G in place), then the inverse column by column
    for (int j = 0; j < nf; ++j) {
        double d = A[(size_t)j * nf + j];
        for (int k = 0; k < j; ++k) d -= A[(size_t)j * nf + k] * A[(size_t)j * nf + k];
        if (!(d > 1e-12 * C.h2inv)) {
            mg_free(P);
            return KHP_OK;
        }
        const double gjj = std::sqrt(d);
        A[(size_t)j * nf + j] = gjj;
        for (int i = j + 1; i < nf; ++i) {
            double v = A[(size_t)i * nf + j];
            for (int k = 0; k < j; ++k) v -= A[(size_t)i * nf + k] * A[(size_t)j * nf + k];
            A[(size_t)i * nf + j] = v / gjj;
        }
    }
    std::vector<double> y(nf);
    for (int c = 0; c < nf; ++c) {
        for (int i = 0; i < nf; ++i) {       // G y = e_c
            double v = i == c ? 1.0 : 0.0;
            for (int k = 0; k < i; ++k) v -= A[(size_t)i * nf + k] * y[k];
            y[i] = v / A[(size_t)i * nf + i];
        }
        for (int i = nf - 1; i >= 0; --i) {  // G^T x = y
            double v = y[i];
            for (int k = i + 1; k < nf; ++k) v -= A[(size_t)k * nf + i] * y[k];
            y[i] = v / A[(size_t)i * nf + i];
        }
        for (int i = 0; i < nf; ++i) inv[(size_t)i * nf + c] = (float)y[i];
    }
    if ((e = cudaMalloc(&P->mg_cinv, sizeof(float) * inv.size())) != cudaSuccess ||
        (e = cudaMalloc(&P->mg_cidx, sizeof(int) * nc)) != cudaSuccess ||
        (e = cudaMemcpyAsync(P->mg_cinv, inv.data(), sizeof(float) * inv.size(), cudaMemcpyHostToDevice,
                             P->stream)) != cudaSuccess ||
        (e = cudaMemcpyAsync(P->mg_cidx, idx.data(), sizeof(int) * nc, cudaMemcpyHostToDevice, P->stream)) !=
            cudaSuccess ||
        (e = cudaStreamSynchronize(P->stream)) != cudaSuccess) {
        mg_free(P);
        return pfail(e == cudaErrorMemoryAllocation ? KHP_ERR_OOM : KHP_ERR_CUDA,
                     std::string("multigrid coarsest level: ") + cudaGetErrorString(e));
    }
    P->mg_nf = nf;
    P->mg_n = L;
    return KHP_OK;
}

bool mg_active(const khp_poisson_s* P) { return P->precond == KHP_POISSON_PRECOND_MULTIGRID && P->mg_n > 0; }

// the V-cycle z = M^-1 r of n right-hand sides (from r's FP32 copy, level
// 0's b) with the block partials of (r.z, r.r)
void mg_vcycle(khp_poisson_s* P, const khp_poisson_s::CGSpace& w, cudaStream_t st, int n) {
    using namespace khp::poisson;
    const int L = P->mg_n;
    for (int l = 0; l + 1 < L; ++l) {
        const Geo f = mg_geo(P, l), c = mg_geo(P, l + 1);
        mg_presmooth_kernel<<<dim3(mg_blocks(f.np, P->sblk), n), kT, 0, st>>>(f, w.mb[l], w.mv[l]);
        mg_restrict_kernel<<<dim3(mg_blocks(8 * c.np, P->sblk), n), kT, 0, st>>>(f, w.mv[l], w.mb[l], c,
                                                                                 w.mb[l + 1]);
    }
    mg_coarse_kernel<<<n, kT, 0, st>>>(mg_geo(P, L - 1), w.mb[L - 1], w.mv[L - 1], P->mg_cinv, P->mg_cidx,
                                       P->mg_nf);
    for (int l = L - 2; l >= 0; --l) {
        const Geo f = mg_geo(P, l), c = mg_geo(P, l + 1);
        const dim3 grid(mg_blocks(f.np, P->sblk), n);
        mg_smooth_kernel<true, false>
            <<<grid, kT, 0, st>>>(f, w.mv[l], c, w.mv[l + 1], w.mb[l], w.mu[l], nullptr, nullptr, nullptr);
        if (l == 0)      // block partials: the CG's block count
            mg_smooth_kernel<false, true>
                <<<dim3(P->nblk, n), kT, 0, st>>>(f, w.mu[0], c, nullptr, w.mb[0], nullptr, w.r, w.z, w.partial);
        else
            mg_smooth_kernel<false, false>
                <<<grid, kT, 0, st>>>(f, w.mu[l], c, nullptr, w.mb[l], w.mv[l], nullptr, nullptr, nullptr);
    }
    if (L == 1) mg_out_kernel<<<dim3(P->nblk, n), kT, 0, st>>>(geo(P), w.mv[0], w.r, w.z, w.partial);
}

// Host side of the tall-skinny QR: fold the blocks' factors into one
// R = [[R11, r12], [0, r22]] of [dF | F] by Givens rotations, then
// gamma = pinv(R11) r12 through a one-sided Jacobi SVD of R11 (the
// singular values of R11 are those of dF); singular values at or below
// eps max(Np, m) sigma_max count as zero, the cutoff of LAPACK's
// minimum-norm least squares.  A zero history gives gamma = 0, the plain
// damped step.
void anderson_solve(const double* factors, int nblk, int m, long long np, double* gamma) {
    constexpr int D = khp::poisson::kMaxDepth + 1;
    const int C = m + 1;
    const int K = C * (C + 1) / 2;
    double R[D][D] = {};
    for (int b = 0; b < nblk; ++b) {
        const double* Q = factors + (size_t)b * K;
        for (int k = 0; k < C; ++k) {
            double a[D] = {};
            for (int j = k; j < C; ++j) a[j] = Q[khp::poisson::tri_at(C, k) + j - k];
            for (int i = 0; i < C; ++i) {
                const double y = a[i];
                if (y == 0.0) continue;
                const double x = R[i][i];
                const double r = std::hypot(x, y);
                const double c = x / r, sn = y / r;
                R[i][i] = r;
                for (int j = i + 1; j < C; ++j) {
                    const double rj = R[i][j];
                    R[i][j] = c * rj + sn * a[j];
                    a[j] = c * a[j] - sn * rj;
                }
            }
        }
    }
    // one-sided Jacobi on the columns of A = R11: A V = U diag(sigma)
    double A[D][D], V[D][D];
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < m; ++j) {
            A[i][j] = R[i][j];
            V[i][j] = i == j ? 1.0 : 0.0;
        }
    for (int sweep = 0; sweep < 80; ++sweep) {
        bool rotated = false;
        for (int p = 0; p < m; ++p)
            for (int q = p + 1; q < m; ++q) {
                double al = 0.0, be = 0.0, ga = 0.0;
                for (int i = 0; i < m; ++i) {
                    al += A[i][p] * A[i][p];
                    be += A[i][q] * A[i][q];
                    ga += A[i][p] * A[i][q];
                }
                if (ga == 0.0 || std::fabs(ga) <= DBL_EPSILON * std::sqrt(al * be)) continue;
                rotated = true;
                const double zeta = (be - al) / (2.0 * ga);
                const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (std::fabs(zeta) + std::sqrt(1.0 + zeta * zeta));
                const double c = 1.0 / std::sqrt(1.0 + t * t), sn = c * t;
                for (int i = 0; i < m; ++i) {
                    const double ap = A[i][p], aq = A[i][q];
                    A[i][p] = c * ap - sn * aq;
                    A[i][q] = sn * ap + c * aq;
                    const double vp = V[i][p], vq = V[i][q];
                    V[i][p] = c * vp - sn * vq;
                    V[i][q] = sn * vp + c * vq;
                }
            }
        if (!rotated) break;
    }
    double sig[D], smax = 0.0;
    for (int j = 0; j < m; ++j) {
        double t = 0.0;
        for (int i = 0; i < m; ++i) t += A[i][j] * A[i][j];
        sig[j] = std::sqrt(t);
        smax = std::max(smax, sig[j]);
    }
    const double cut = DBL_EPSILON * (double)std::max<long long>(np, m) * smax;
    for (int i = 0; i < m; ++i) gamma[i] = 0.0;
    for (int j = 0; j < m; ++j) {
        if (!(sig[j] > cut) || !std::isfinite(sig[j])) continue;
        double ur = 0.0;                   // u_j . r12 with u_j = A[:, j] / sigma_j
        for (int i = 0; i < m; ++i) ur += A[i][j] * R[i][m];
        const double w = ur / (sig[j] * sig[j]);
        for (int i = 0; i < m; ++i) gamma[i] += V[i][j] * w;
    }
    for (int i = 0; i < m; ++i)
        if (!std::isfinite(gamma[i])) {
            for (int k = 0; k < m; ++k) gamma[k] = 0.0;
            break;
        }
}

}  // namespace

extern "C" {

khp_status khp_poisson_create(khp_poisson* out, int nx, int ny, int nz, double h_nm, double eps_r,
                              const uint8_t* gate_mask_dev, const double* gate_phi_dev, void* stream) {
    khp_set_error(KHP_OK, "");
    if (!out) return pfail(KHP_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (nx < 1 || ny < 1 || nz < 1) return pfail(KHP_ERR_INVALID_ARG, "grid sizes must be >= 1");
    if (!(h_nm > 0.0) || !std::isfinite(h_nm)) return pfail(KHP_ERR_INVALID_ARG, "h must be > 0");
    if (!(eps_r > 0.0) || !std::isfinite(eps_r)) return pfail(KHP_ERR_INVALID_ARG, "eps_r must be > 0");
    if (!gate_mask_dev || !gate_phi_dev) return pfail(KHP_ERR_INVALID_ARG, "gate mask or gate potential is NULL");
    const long long np = (long long)nx * ny * nz;
    if (np > (1LL << 31)) return pfail(KHP_ERR_INVALID_ARG, "grid too large");
    khp_poisson_s* P = new khp_poisson_s();
    std::memset(P, 0, sizeof(*P));
    P->nx = nx; P->ny = ny; P->nz = nz; P->np = np; P->h = h_nm; P->eps_r = eps_r;
    // e / (eps0 eps_r) in V nm
    P->coef = 1.602176634e-19 / (8.8541878128e-21 * eps_r);
    P->h2inv = 1.0 / (h_nm * h_nm);
    P->stream = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) {
        delete P;
        return pfail(KHP_ERR_CUDA, "no CUDA device");
    }
    P->nblk = (int)std::min<long long>((np + kT - 1) / kT, 2LL * sms);
    P->sblk = (int)std::min<long long>((np + kT - 1) / kT, 8LL * sms);
    cudaError_t e = cudaSuccess;
    const size_t vb = sizeof(double) * np;
    if ((e = cudaMalloc(&P->gate, np)) != cudaSuccess || (e = cudaMalloc(&P->code, sizeof(uint16_t) * np)) != cudaSuccess ||
        (e = cudaMalloc(&P->gphi, vb)) != cudaSuccess ||
        (e = cudaStreamCreateWithFlags(&P->work, cudaStreamNonBlocking)) != cudaSuccess) {
        free_all(P);
        delete P;
        return pfail(e == cudaErrorMemoryAllocation ? KHP_ERR_OOM : KHP_ERR_CUDA,
                     std::string("allocation: ") + cudaGetErrorString(e));
    }
    if ((e = cudaMemcpyAsync(P->gate, gate_mask_dev, np, cudaMemcpyDeviceToDevice, P->stream)) != cudaSuccess) {
        free_all(P);
        delete P;
        return pfail(KHP_ERR_CUDA, std::string("gate copy: ") + cudaGetErrorString(e));
    }
    khp::poisson::copy_gate_values_kernel<<<P->nblk, kT, 0, P->stream>>>(np, P->gate, gate_phi_dev, P->gphi);
    khp::poisson::mg_code_kernel<<<P->nblk, kT, 0, P->stream>>>(geo(P), P->code);
    if ((e = cudaGetLastError()) != cudaSuccess || (e = cudaStreamSynchronize(P->stream)) != cudaSuccess) {
        free_all(P);
        delete P;
        return pfail(KHP_ERR_CUDA, std::string("gate set-up: ") + cudaGetErrorString(e));
    }
    P->precond = KHP_POISSON_PRECOND_MULTIGRID;
    const khp_status ms = mg_build(P);
    if (ms != KHP_OK) {
        free_all(P);
        delete P;
        return ms;
    }
    if ((e = space_alloc(P, P->one, 1)) != cudaSuccess) {
        free_all(P);
        delete P;
        return pfail(e == cudaErrorMemoryAllocation ? KHP_ERR_OOM : KHP_ERR_CUDA,
                     std::string("CG vectors: ") + cudaGetErrorString(e));
    }
    *out = P;
    return KHP_OK;
}

// one CG iteration of n right-hand sides: 5 launches with the Jacobi
// preconditioner, the V-cycle's in place of the z = r / diag step with the
// multigrid one
static void cg_iteration(khp_poisson_s* P, const khp_poisson_s::CGSpace& w, const khp::poisson::Geo& g,
                         cudaStream_t st, int n) {
    using namespace khp::poisson;
    const int nb = P->nblk;
    const dim3 grid(nb, n);              // kernels with block partials
    const dim3 sgrid(P->sblk, n);        // streaming kernels
    apply_kernel<<<grid, kT, 0, st>>>(g, w.p, w.Ap, w.partial);
    finish_kernel<<<n, kT, 0, st>>>(w.partial, nb, 2, w.s);
    if (mg_active(P)) {
        update_mg_kernel<<<sgrid, kT, 0, st>>>(g, w.s, w.p, w.Ap, w.x, w.r, w.mb[0]);
        mg_vcycle(P, w, st, n);
    } else {
        update_kernel<<<grid, kT, 0, st>>>(g, w.s, w.p, w.Ap, w.x, w.r, w.z, w.partial);
    }
    finish_kernel<<<n, kT, 0, st>>>(w.partial, nb, 3, w.s);
    direction_kernel<<<sgrid, kT, 0, st>>>(g, w.s, w.z, w.p);
}

// CG solves of A phi_k = coef * rho_scale * rho_k (free points) for the n
// right-hand sides of w (rho_k at rho_dev + k ld_rho, phi_k at phi_dev +
// k ld_phi) with the gate potentials gphi (the handle's, or zeros for
// grounded gates); phi_k is the start at the free points and the solution
// on return.  All right-hand sides iterate until the largest relative
// residual is at most tol.  Synchronous.
static khp_status cg_solve(khp_poisson P, khp_poisson_s::CGSpace& w, int n, const double* rho_dev,
                           long long ld_rho, double rho_scale, const double* gphi, double* phi_dev,
                           long long ld_phi, double tol, int max_iter, int* iterations, double* rel_residual) {
    using namespace khp::poisson;
    const Geo g = geo(P);
    const int nb = P->nblk;
    const dim3 grid(nb, n);
    // the caller's work (rho, phi) is complete before the private stream starts
    PCK(cudaStreamSynchronize(P->stream));
    cudaStream_t st = P->work;
    double* hp = w.host;
    rhs_kernel<<<grid, kT, 0, st>>>(g, rho_dev, ld_rho, gphi, P->coef * rho_scale, phi_dev, ld_phi, w.b, w.x,
                                    w.partial);
    finish_kernel<<<n, kT, 0, st>>>(w.partial, nb, 0, w.s);
    apply_kernel<<<grid, kT, 0, st>>>(g, w.x, w.Ap, w.partial);
    const bool mg = mg_active(P);
    if (mg) {
        init_mg_kernel<<<dim3(P->sblk, n), kT, 0, st>>>(g, w.b, w.Ap, w.r, w.mb[0]);
        mg_vcycle(P, w, st, n);
    } else {
        init_kernel<<<grid, kT, 0, st>>>(g, w.b, w.Ap, w.r, w.z, w.p, w.partial);
    }
    finish_kernel<<<n, kT, 0, st>>>(w.partial, nb, 1, w.s);
    PCKL("CG set-up launches");
    if (mg) PCK(cudaMemcpyAsync(w.p, w.z, sizeof(double) * P->np * n, cudaMemcpyDeviceToDevice, st));
    // the largest relative residual over the right-hand sides (a zero
    // right-hand side counts its absolute residual, zero from a zero start)
    auto worst = [&]() {
        double m = 0.0;
        for (int k = 0; k < n; ++k) {
            const double bb = hp[8 * k + 5], rr = hp[8 * k + 4];
            const double rel = bb > 0.0 ? std::sqrt(rr / bb) : std::sqrt(rr);
            m = std::isnan(rel) ? rel : std::max(m, rel);
            if (std::isnan(m)) break;
        }
        return m;
    };
    PCK(cudaMemcpyAsync(hp, w.s, sizeof(double) * 8 * n, cudaMemcpyDeviceToHost, st));
    PCK(cudaStreamSynchronize(st));
    double rel = worst();
    if (!std::isfinite(rel)) return pfail(KHP_ERR_BREAKDOWN, "Poisson CG: non-finite initial residual");
    int it = 0;
    // residual check every 16 Jacobi-preconditioned iterations or every 8
    // multigrid ones (the graph holds the iterations between two checks)
    const int per_check = mg ? 8 : 16;
    while (rel > tol && it < max_iter) {
        const int chunk = std::min(per_check, max_iter - it);
        if (chunk == per_check) {
            if (w.have_chunk && w.chunk_n != n) {
                cudaGraphExecDestroy(w.chunk);
                w.have_chunk = false;
            }
            if (!w.have_chunk) {
                cudaGraph_t graph;
                PCK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
                for (int k = 0; k < per_check; ++k) cg_iteration(P, w, g, st, n);
                PCK(cudaStreamEndCapture(st, &graph));
                const cudaError_t e = cudaGraphInstantiate(&w.chunk, graph, 0);
                cudaGraphDestroy(graph);
                PCK(e);
                w.have_chunk = true;
                w.chunk_n = n;
            }
            PCK(cudaGraphLaunch(w.chunk, st));
        } else {
            for (int k = 0; k < chunk; ++k) cg_iteration(P, w, g, st, n);
        }
        PCKL("CG iterations");
        it += chunk;
        PCK(cudaMemcpyAsync(hp, w.s, sizeof(double) * 8 * n, cudaMemcpyDeviceToHost, st));
        PCK(cudaStreamSynchronize(st));
        rel = worst();
        if (!std::isfinite(rel)) return pfail(KHP_ERR_BREAKDOWN, "Poisson CG produced a non-finite residual");
    }
    output_kernel<<<dim3(P->sblk, n), kT, 0, st>>>(g, w.x, gphi, phi_dev, ld_phi);
    PCKL("CG output");
    PCK(cudaStreamSynchronize(st));
    if (iterations) *iterations = it;
    if (rel_residual) *rel_residual = rel;
    if (rel > tol) return pfail(KHP_ERR_NOT_CONVERGED, "Poisson CG reached max_iter");
    return KHP_OK;
}

static khp_status ensure_zeros(khp_poisson P) {
    if (P->r_zero) return KHP_OK;
    cudaError_t e;
    if ((e = cudaMalloc(&P->r_zero, sizeof(double) * P->np)) != cudaSuccess)
        return pfail(KHP_ERR_OOM, std::string("zero gate potentials: ") + cudaGetErrorString(e));
    PCK(cudaMemsetAsync(P->r_zero, 0, sizeof(double) * P->np, P->work));
    PCK(cudaStreamSynchronize(P->work));
    return KHP_OK;
}

// nrhs solves (contiguous [nrhs][Np] rho and phi, rho scaled by rho_scale)
// in batches of at most kMaxRhs right-hand sides on the handle's second CG
// space; iterations = the most any batch took, rel = the largest residual
static khp_status cg_solve_batches(khp_poisson P, const double* rho_dev, double rho_scale, const double* gphi,
                                   double* phi_dev, int nrhs, double tol, int max_iter, int* iterations,
                                   double* rel_residual) {
    const int cap = std::min(nrhs, khp_poisson_s::kMaxRhs);
    if (P->many.cap < cap) {
        const cudaError_t e = space_alloc(P, P->many, cap);
        if (e != cudaSuccess) {
            space_free(P->many);
            return pfail(e == cudaErrorMemoryAllocation ? KHP_ERR_OOM : KHP_ERR_CUDA,
                         std::string("CG vectors of a batch: ") + cudaGetErrorString(e));
        }
    }
    int it_max = 0;
    double rel_max = 0.0;
    khp_status st = KHP_OK;
    for (int k0 = 0; k0 < nrhs && st == KHP_OK; k0 += cap) {
        const int n = std::min(cap, nrhs - k0);
        int it = 0;
        double rel = 0.0;
        st = cg_solve(P, P->many, n, rho_dev + (size_t)k0 * P->np, P->np, rho_scale, gphi,
                      phi_dev + (size_t)k0 * P->np, P->np, tol, max_iter, &it, &rel);
        it_max = std::max(it_max, it);
        rel_max = std::max(rel_max, rel);
    }
    if (iterations) *iterations = it_max;
    if (rel_residual) *rel_residual = rel_max;
    return st;
}

khp_status khp_poisson_solve(khp_poisson P, const double* rho_dev, double* phi_dev, double tol, int max_iter,
                             int* iterations, double* rel_residual) {
    khp_set_error(KHP_OK, "");
    if (!P) return pfail(KHP_ERR_INVALID_ARG, "handle is NULL");
    if (!rho_dev || !phi_dev) return pfail(KHP_ERR_INVALID_ARG, "rho or phi is NULL");
    if (!(tol > 0.0) || max_iter < 1) return pfail(KHP_ERR_INVALID_ARG, "need tol > 0 and max_iter >= 1");
    return cg_solve(P, P->one, 1, rho_dev, P->np, 1.0, P->gphi, phi_dev, P->np, tol, max_iter, iterations,
                    rel_residual);
}

khp_status khp_poisson_solve_many(khp_poisson P, const double* rho_dev, double* phi_dev, int nrhs, int grounded,
                                  double tol, int max_iter, int* iterations, double* max_rel_residual) {
    khp_set_error(KHP_OK, "");
    if (!P) return pfail(KHP_ERR_INVALID_ARG, "handle is NULL");
    if (!rho_dev || !phi_dev) return pfail(KHP_ERR_INVALID_ARG, "rho or phi is NULL");
    if (nrhs < 1) return pfail(KHP_ERR_INVALID_ARG, "nrhs must be >= 1");
    if (!(tol > 0.0) || max_iter < 1) return pfail(KHP_ERR_INVALID_ARG, "need tol > 0 and max_iter >= 1");
    if (grounded) CKSP(ensure_zeros(P));
    return cg_solve_batches(P, rho_dev, 1.0, grounded ? P->r_zero : P->gphi, phi_dev, nrhs, tol, max_iter,
                            iterations, max_rel_residual);
}

khp_status khp_sp_update(khp_poisson P, const double* V_ext_dev, const double* phi_dev, double mix, double* V_dev,
                         double* max_change) {
    khp_set_error(KHP_OK, "");
    if (!P) return pfail(KHP_ERR_INVALID_ARG, "handle is NULL");
    if (!phi_dev || !V_dev) return pfail(KHP_ERR_INVALID_ARG, "phi or V is NULL");
    if (!(mix > 0.0 && mix <= 1.0)) return pfail(KHP_ERR_INVALID_ARG, "mix must be in (0, 1]");
    using namespace khp::poisson;
    PCK(cudaStreamSynchronize(P->stream));
    mix_kernel<<<P->nblk, kT, 0, P->work>>>(P->np, V_ext_dev, phi_dev, mix, V_dev, P->one.partial);
    max_finish_kernel<<<1, kT, 0, P->work>>>(P->one.partial, P->nblk, P->one.s + 6);
    PCKL("linear update");
    PCK(cudaMemcpyAsync(P->one.host + 6, P->one.s + 6, sizeof(double), cudaMemcpyDeviceToHost, P->work));
    PCK(cudaStreamSynchronize(P->work));
    if (max_change) *max_change = P->one.host[6];
    return KHP_OK;
}

khp_status khp_sp_anderson(khp_poisson P, const double* V_ext_dev, const double* phi_dev, double beta, int depth,
                           double* V_dev, double* max_change) {
    khp_set_error(KHP_OK, "");
    using namespace khp::poisson;
    if (!P) return pfail(KHP_ERR_INVALID_ARG, "handle is NULL");
    if (!phi_dev || !V_dev) return pfail(KHP_ERR_INVALID_ARG, "phi or V is NULL");
    if (!(beta > 0.0 && beta <= 1.0)) return pfail(KHP_ERR_INVALID_ARG, "beta must be in (0, 1]");
    if (depth < 1 || depth > kMaxDepth) return pfail(KHP_ERR_INVALID_ARG, "depth out of range 1..8");
    const long long np = P->np;
    if (!P->a_dv) {
        cudaError_t e;
        if ((e = cudaMalloc(&P->a_dv, sizeof(double) * kMaxDepth * np)) != cudaSuccess ||
            (e = cudaMalloc(&P->a_df, sizeof(double) * kMaxDepth * np)) != cudaSuccess ||
            (e = cudaMalloc(&P->a_vprev, sizeof(double) * np)) != cudaSuccess ||
            (e = cudaMalloc(&P->a_fprev, sizeof(double) * np)) != cudaSuccess ||
            (e = cudaMalloc(&P->a_f, sizeof(double) * np)) != cudaSuccess ||
            (e = cudaMalloc(&P->a_partial, sizeof(double) * kMaxR * P->nblk)) != cudaSuccess ||
            (e = cudaMallocHost(&P->a_host, sizeof(double) * kMaxR * P->nblk)) != cudaSuccess)
            return pfail(KHP_ERR_OOM, std::string("Anderson history: ") + cudaGetErrorString(e));
        P->a_count = 0;
        P->a_depth = depth;
    }
    if (depth != P->a_depth) {            // a new depth starts a new history
        P->a_count = 0;
        P->a_depth = depth;
    }
    PCK(cudaStreamSynchronize(P->stream));
    cudaStream_t st = P->work;
    const int nb = P->nblk;
    // the newest differences go to ring slot (count - 1) % depth
    double* dv = nullptr;
    double* df = nullptr;
    if (P->a_count > 0) {
        const int slot = (P->a_count - 1) % depth;
        dv = P->a_dv + (size_t)slot * np;
        df = P->a_df + (size_t)slot * np;
    }
    anderson_residual_kernel<<<nb, kT, 0, st>>>(np, V_ext_dev, phi_dev, V_dev, P->a_f, P->a_vprev, P->a_fprev, dv,
                                                df);
    PCKL("Anderson residual");
    const int m = std::min(P->a_count, depth);
    AndersonCoef c{};
    if (m > 0) {
        const int K = (m + 1) * (m + 2) / 2;
        switch (m) {
#define KHP_AQ(M) case M: anderson_qr_kernel<M><<<nb, kT, 0, st>>>(np, P->a_df, P->a_f, P->a_partial); break;
            KHP_AQ(1) KHP_AQ(2) KHP_AQ(3) KHP_AQ(4) KHP_AQ(5) KHP_AQ(6) KHP_AQ(7) KHP_AQ(8)
#undef KHP_AQ
        }
        PCKL("Anderson QR");
        PCK(cudaMemcpyAsync(P->a_host, P->a_partial, sizeof(double) * K * nb, cudaMemcpyDeviceToHost, st));
        PCK(cudaStreamSynchronize(st));
        anderson_solve(P->a_host, nb, m, np, c.gamma);
    }
    anderson_update_kernel<<<nb, kT, 0, st>>>(np, m, beta, c, V_dev, P->a_f, P->a_dv, P->a_df, P->one.partial);
    max_finish_kernel<<<1, kT, 0, st>>>(P->one.partial, nb, P->one.s + 6);
    PCKL("Anderson update");
    PCK(cudaMemcpyAsync(P->one.host + 6, P->one.s + 6, sizeof(double), cudaMemcpyDeviceToHost, st));
    PCK(cudaStreamSynchronize(st));
    P->a_count += 1;
    if (max_change) *max_change = P->one.host[6];
    return KHP_OK;
}

// Fermi level of the SP loop's occupations (Sec. II B; host only).  The
// hole count N(mu) = sum_i f((E_i - mu) / kT), f(x) = 1 / (1 + e^x), rises
// monotonically in mu with slope N'(mu) = sum_i f (1 - f) / kT.  Newton's
// method on N(mu) = n_holes, kept inside a bracket [lo, hi] that every
// evaluation narrows (N < n_holes moves lo up, N > n_holes moves hi down);
// a Newton step that leaves the bracket, or stalls on a flat stretch of N
// between well separated levels, is replaced by the bracket's midpoint.
// E finite, 0 < n_holes < n, kT > 0 (checked by the callers).
static double fd_occ(double e, double mu, double kT) {
    const double x = (e - mu) / kT;
    if (x >= 0.0) {
        const double t = std::exp(-x);
        return t / (1.0 + t);
    }
    return 1.0 / (1.0 + std::exp(x));
}

static double fermi_solve(const double* E_host, int n, double n_holes, double kT, double* occ_host) {
    double emin = E_host[0], emax = E_host[0];
    for (int i = 0; i < n; ++i) {
        emin = std::min(emin, E_host[i]);
        emax = std::max(emax, E_host[i]);
    }
    // N(lo) <= n e^-(L) < n_holes and N(hi) >= n - n e^-(L) > n_holes
    const double L = std::log((double)n) + 60.0 + std::fabs(std::log(std::min(n_holes, n - n_holes)));
    double lo = emin - L * kT, hi = emax + L * kT;
    double mu = 0.5 * (lo + hi), dx = hi - lo, dxold = dx;
    for (int it = 0; it < 400; ++it) {
        double N = 0.0, dN = 0.0;
        for (int i = 0; i < n; ++i) {
            const double f = fd_occ(E_host[i], mu, kT);
            N += f;
            dN += f * (1.0 - f);
        }
        dN /= kT;
        const double r = N - n_holes;
        if (r == 0.0) break;
        if (r < 0.0) lo = mu; else hi = mu;
        const double newton = dN > 0.0 ? mu - r / dN : lo;
        // bisect when Newton leaves the bracket or would not halve the
        // step of the iteration before last
        const bool bisect = !(newton > lo && newton < hi) || std::fabs(2.0 * r) > std::fabs(dxold * dN);
        dxold = dx;
        const double prev = mu;
        mu = bisect ? 0.5 * (lo + hi) : newton;
        dx = mu - prev;
        if (std::fabs(dx) <= 2.0 * DBL_EPSILON * std::max(std::fabs(mu), kT)) break;
    }
    if (occ_host)
        for (int i = 0; i < n; ++i) occ_host[i] = fd_occ(E_host[i], mu, kT);
    return mu;
}

khp_status khp_fermi_level(const double* E_host, int n, double n_holes, double kT, double* mu_out,
                           double* occ_host) {
    khp_set_error(KHP_OK, "");
    if (!E_host || !mu_out) return pfail(KHP_ERR_INVALID_ARG, "E or mu is NULL");
    if (n < 1) return pfail(KHP_ERR_INVALID_ARG, "n must be >= 1");
    if (!(kT > 0.0) || !std::isfinite(kT)) return pfail(KHP_ERR_INVALID_ARG, "kT must be > 0");
    if (!(n_holes > 0.0 && n_holes < n)) return pfail(KHP_ERR_INVALID_ARG, "n_holes must lie in (0, n)");
    for (int i = 0; i < n; ++i)
        if (!std::isfinite(E_host[i])) return pfail(KHP_ERR_INVALID_ARG, "non-finite level");
    *mu_out = fermi_solve(E_host, n, n_holes, kT, occ_host);
    return KHP_OK;
}

// Occupations relaxed in a fixed set of states (host, n <= 64): the
// effective levels eps solve eps = e0 + K f(eps), f the Fermi-Dirac
// occupations at the Fermi level of eps (fermi_solve).  Newton's method on
// R(eps) = eps - e0 - K f(eps) with the Jacobian I + K B / kT,
// B = diag(s) - s s^T / sum(s), s = f (1 - f) (the derivative of f at a
// fixed hole number); the step is halved until |R| falls.  Gaussian
// elimination with partial pivoting for the n x n system.
static bool relax_newton(const double* e0, const double* K, int n, double n_holes, double kT, double* f,
                         double* mu) {
    std::vector<double> eps(n), R(n), J((size_t)n * n), step(n), trial(n), f2(n);
    auto residual = [&](const std::vector<double>& e, double* ff, std::vector<double>& r) {
        const double m = fermi_solve(e.data(), n, n_holes, kT, ff);
        double nr = 0.0;
        for (int i = 0; i < n; ++i) {
            double v = e[i] - e0[i];
            for (int j = 0; j < n; ++j) v -= K[(size_t)i * n + j] * ff[j];
            r[i] = v;
            nr += v * v;
        }
        return std::make_pair(m, std::sqrt(nr));
    };
    // start: the levels shifted by the occupations of the unshifted levels
    {
        std::vector<double> e(e0, e0 + n);
        fermi_solve(e.data(), n, n_holes, kT, f);
        for (int i = 0; i < n; ++i) {
            double v = e0[i];
            for (int j = 0; j < n; ++j) v += K[(size_t)i * n + j] * f[j];
            eps[i] = v;
        }
    }
    for (int it = 0; it < 200; ++it) {
        auto [m, nr] = residual(eps, f, R);
        *mu = m;
        double emax = 1e-3;
        for (int i = 0; i < n; ++i) emax = std::max(emax, std::fabs(eps[i]));
        if (nr <= 1e-15 * emax) return true;
        double S = 0.0;
        std::vector<double> sv(n);
        for (int i = 0; i < n; ++i) {
            sv[i] = f[i] * (1.0 - f[i]);
            S += sv[i];
        }
        // J = I + K B / kT, B_lj = s_l delta_lj - s_l s_j / S
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) {
                double v = K[(size_t)i * n + j] * sv[j];
                if (S > 0.0) {
                    double ks = 0.0;
                    for (int l = 0; l < n; ++l) ks += K[(size_t)i * n + l] * sv[l];
                    v -= ks * sv[j] / S;
                }
                J[(size_t)i * n + j] = (i == j ? 1.0 : 0.0) + v / kT;
            }
        for (int i = 0; i < n; ++i) step[i] = -R[i];
        for (int c = 0; c < n; ++c) {      // elimination with partial pivoting
            int piv = c;
            for (int r = c + 1; r < n; ++r)
                if (std::fabs(J[(size_t)r * n + c]) > std::fabs(J[(size_t)piv * n + c])) piv = r;
            if (!(J[(size_t)piv * n + c] != 0.0)) return false;
            if (piv != c) {
                for (int k = 0; k < n; ++k) std::swap(J[(size_t)c * n + k], J[(size_t)piv * n + k]);
                std::swap(step[c], step[piv]);
            }
            for (int r = c + 1; r < n; ++r) {
                const double t = J[(size_t)r * n + c] / J[(size_t)c * n + c];
                for (int k = c; k < n; ++k) J[(size_t)r * n + k] -= t * J[(size_t)c * n + k];
                step[r] -= t * step[c];
            }
        }
        for (int c = n - 1; c >= 0; --c) {
            double v = step[c];
            for (int k = c + 1; k < n; ++k) v -= J[(size_t)c * n + k] * step[k];
            step[c] = v / J[(size_t)c * n + c];
        }
        double a = 1.0;
        std::vector<double> R2(n);
        while (true) {
            for (int i = 0; i < n; ++i) trial[i] = eps[i] + a * step[i];
            const double nr2 = residual(trial, f2.data(), R2).second;
            if (nr2 < nr * (1.0 - 1e-4 * a) || a < 1e-12) break;
            a *= 0.5;
        }
        eps = trial;
    }
    *mu = fermi_solve(eps.data(), n, n_holes, kT, f);
    return true;
}

khp_status khp_sp_relax_occupations(khp_poisson P, const double* dens_dev, const double* E_host, int n,
                                    double n_holes, double kT_ev, const double* V_dev, const double* V_ext_dev,
                                    double* phi_dev, double tol, double* occ_host, double* mu_out) {
    khp_set_error(KHP_OK, "");
    using namespace khp::poisson;
    if (!P) return pfail(KHP_ERR_INVALID_ARG, "handle is NULL");
    if (!dens_dev || !E_host || !V_dev || !phi_dev) return pfail(KHP_ERR_INVALID_ARG, "NULL argument");
    if (n < 1 || n > KHP_MAX_M) return pfail(KHP_ERR_INVALID_ARG, "n out of range 1..64");
    if (!(kT_ev > 0.0) || !std::isfinite(kT_ev)) return pfail(KHP_ERR_INVALID_ARG, "kT must be > 0");
    if (!(n_holes > 0.0 && n_holes < n)) return pfail(KHP_ERR_INVALID_ARG, "n_holes must lie in (0, n)");
    if (!(tol > 0.0)) return pfail(KHP_ERR_INVALID_ARG, "tol must be > 0");
    for (int i = 0; i < n; ++i)
        if (!std::isfinite(E_host[i])) return pfail(KHP_ERR_INVALID_ARG, "non-finite level");
    const long long np = P->np;
    const int nb = P->nblk;
    const int nch = (n + kRJ - 1) / kRJ;
    if (!P->r_Q || P->r_nmax < n) {
        if (P->r_Q) cudaFree(P->r_Q);
        P->r_Q = nullptr;
        P->r_nq = 0;
        cudaError_t e;
        if ((e = cudaMalloc(&P->r_Q, sizeof(double) * (size_t)n * np)) != cudaSuccess)
            return pfail(KHP_ERR_OOM, std::string("relaxed step buffers: ") + cudaGetErrorString(e));
        P->r_nmax = n;
    }
    if (!P->r_phig) {
        const int rows = KHP_MAX_M * ((KHP_MAX_M + kRJ - 1) / kRJ);
        cudaError_t e;
        CKSP(ensure_zeros(P));
        if ((e = cudaMalloc(&P->r_phig, sizeof(double) * np)) != cudaSuccess ||
            (e = cudaMalloc(&P->r_partial, sizeof(double) * (size_t)rows * nb * (kRJ + 1))) != cudaSuccess ||
            (e = cudaMalloc(&P->r_out, sizeof(double) * (size_t)rows * (kRJ + 1))) != cudaSuccess ||
            (e = cudaMallocHost(&P->r_host, sizeof(double) * (size_t)rows * (kRJ + 1))) != cudaSuccess)
            return pfail(KHP_ERR_OOM, std::string("relaxed step buffers: ") + cudaGetErrorString(e));
        PCK(cudaMemsetAsync(P->r_phig, 0, sizeof(double) * np, P->work));
        PCK(cudaStreamSynchronize(P->work));
        P->r_have_phig = false;
    }
    const int max_iter = 100000;
    if (!P->r_have_phig) {
        CKSP(cg_solve(P, P->one, 1, P->r_zero, np, 1.0, P->gphi, P->r_phig, np, tol, max_iter, nullptr, nullptr));
        P->r_have_phig = true;
    }
    // unit-occupation potentials (grounded gates), solved together, each
    // started from the previous call's solution for the same state index
    if (P->r_nq < n) {
        PCK(cudaMemsetAsync(P->r_Q + (size_t)P->r_nq * np, 0, sizeof(double) * (size_t)(n - P->r_nq) * np, P->work));
        PCK(cudaStreamSynchronize(P->work));
    }
    const double h3inv = 1.0 / (P->h * P->h * P->h);
    CKSP(cg_solve_batches(P, dens_dev, h3inv, P->r_zero, P->r_Q, n, tol, max_iter, nullptr, nullptr));
    P->r_nq = std::max(P->r_nq, n);
    cudaStream_t st = P->work;
    relax_dots_kernel<<<dim3(nb, n, nch), kT, 0, st>>>(np, n, dens_dev, P->r_Q, P->r_phig, V_dev, V_ext_dev,
                                                       P->r_partial);
    relax_sum_kernel<<<n * nch, 32, 0, st>>>(P->r_partial, nb, P->r_out);
    PCKL("relaxed step: sums");
    PCK(cudaMemcpyAsync(P->r_host, P->r_out, sizeof(double) * (size_t)n * nch * (kRJ + 1), cudaMemcpyDeviceToHost, st));
    PCK(cudaStreamSynchronize(st));
    std::vector<double> K((size_t)n * n), e0(n), f(n);
    for (int i = 0; i < n; ++i) {
        for (int j = 0; j < n; ++j) K[(size_t)i * n + j] = P->r_host[((size_t)i * nch + j / kRJ) * (kRJ + 1) + j % kRJ];
        e0[i] = E_host[i] + P->r_host[((size_t)i * nch) * (kRJ + 1) + kRJ];
    }
    for (int i = 0; i < n; ++i)          // symmetric by reciprocity: average the rounding
        for (int j = i + 1; j < n; ++j) {
            const double v = 0.5 * (K[(size_t)i * n + j] + K[(size_t)j * n + i]);
            K[(size_t)i * n + j] = K[(size_t)j * n + i] = v;
        }
    double mu = 0.0;
    if (!relax_newton(e0.data(), K.data(), n, n_holes, kT_ev, f.data(), &mu))
        return pfail(KHP_ERR_BREAKDOWN, "relaxed occupations: singular Newton system");
    RelaxCoef c{};
    for (int j = 0; j < n; ++j) c.f[j] = f[j];
    relax_combine_kernel<<<nb, kT, 0, st>>>(np, n, c, P->r_phig, P->r_Q, phi_dev);
    PCKL("relaxed step: potential");
    PCK(cudaStreamSynchronize(st));
    if (occ_host)
        for (int j = 0; j < n; ++j) occ_host[j] = f[j];
    if (mu_out) *mu_out = mu;
    return KHP_OK;
}

khp_status khp_poisson_set_preconditioner(khp_poisson P, int kind, int* levels) {
    khp_set_error(KHP_OK, "");
    if (!P) return pfail(KHP_ERR_INVALID_ARG, "handle is NULL");
    if (kind != KHP_POISSON_PRECOND_JACOBI && kind != KHP_POISSON_PRECOND_MULTIGRID)
        return pfail(KHP_ERR_INVALID_ARG, "unknown preconditioner");
    if (kind != P->precond) {
        PCK(cudaStreamSynchronize(P->work));
        for (khp_poisson_s::CGSpace* w : {&P->one, &P->many})
            if (w->have_chunk) {
                cudaGraphExecDestroy(w->chunk);
                w->have_chunk = false;
            }
    }
    P->precond = kind;
    if (levels) *levels = mg_active(P) ? P->mg_n : 0;
    return KHP_OK;
}

khp_status khp_sp_anderson_reset(khp_poisson P) {
    khp_set_error(KHP_OK, "");
    if (!P) return pfail(KHP_ERR_INVALID_ARG, "handle is NULL");
    P->a_count = 0;
    return KHP_OK;
}

khp_status khp_poisson_destroy(khp_poisson P) {
    if (!P) return KHP_OK;
    cudaStreamSynchronize(P->stream);
    if (P->work) cudaStreamSynchronize(P->work);
    free_all(P);
    delete P;
    return KHP_OK;
}

}  // extern "C"
