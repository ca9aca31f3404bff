// Shared device helpers and the handle layout of the k.p eigensolver.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "khp.h"

namespace khp {

// ---------------------------------------------------------------- complex
template <typename R> struct cx;
template <> struct cx<double> { using t = double2; };
template <> struct cx<float> { using t = float2; };

template <typename R> using cx_t = typename cx<R>::t;

template <typename R>
__device__ __forceinline__ cx_t<R> mk(R re, R im) { cx_t<R> z; z.x = re; z.y = im; return z; }

// a * b
template <typename C>
__device__ __forceinline__ C cmul(C a, C b) {
    C r; r.x = a.x * b.x - a.y * b.y; r.y = a.x * b.y + a.y * b.x; return r;
}
// conj(a) * b
template <typename C>
__device__ __forceinline__ C cmulc(C a, C b) {
    C r; r.x = a.x * b.x + a.y * b.y; r.y = a.x * b.y - a.y * b.x; return r;
}
// acc += a * b
template <typename C>
__device__ __forceinline__ void cfma(C& acc, C a, C b) {
    acc.x = fma(a.x, b.x, acc.x); acc.x = fma(-a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y); acc.y = fma(a.y, b.x, acc.y);
}
// acc += conj(a) * b
template <typename C>
__device__ __forceinline__ void cfmac(C& acc, C a, C b) {
    acc.x = fma(a.x, b.x, acc.x); acc.x = fma(a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y); acc.y = fma(-a.y, b.x, acc.y);
}

// packed upper-triangle index k -> (i, j), i <= j, rows of an m x m matrix
// in order: (0,0) (0,1) .. (0,m-1) (1,1) ..
__device__ __forceinline__ void packed_ij(int k, int m, int& i, int& j) {
    int row = 0, len = m;
    while (k >= len) { k -= len; ++row; --len; }
    i = row;
    j = row + k;
}

// ------------------------------------------------------------ stencil data
// The 9 neighbour pairs of the 19-point stencil: pair d couples a point to
// the neighbours at +off[d] and -off[d] with the same real symmetric 3x3
// orbital matrix (the coupling of -delta equals that of +delta).
// d = 0,1,2: faces x, y, z; d = 3..8: edges (xy,+), (xy,-), (xz,+), (xz,-),
// (yz,+), (yz,-) where (ab,+) = e_a + e_b and (ab,-) = e_a - e_b.
__host__ __device__ constexpr int pair_dx(int d) {
    return d == 0 ? 1 : d == 3 ? 1 : d == 4 ? 1 : d == 5 ? 1 : d == 6 ? 1 : 0;
}
__host__ __device__ constexpr int pair_dy(int d) {
    return d == 1 ? 1 : d == 3 ? 1 : d == 4 ? -1 : d == 7 ? 1 : d == 8 ? 1 : 0;
}
__host__ __device__ constexpr int pair_dz(int d) {
    return d == 2 ? 1 : d == 5 ? 1 : d == 6 ? -1 : d == 7 ? 1 : d == 8 ? -1 : 0;
}

// symmetric 3x3 stored as (00, 11, 22, 12, 02, 01); bit k of a nonzero
// mask flags entry k as structurally nonzero (zero entries are skipped)
template <typename R>
struct Coeffs {
    R hop[9][6];        // neighbour-pair orbital matrices
    R soz_re[6][6];     // spin-orbit + Zeeman (constant over the grid)
    R soz_im[6][6];
    unsigned hop_nz[9];     // 6-bit masks
    unsigned onsite_nz;     // 6-bit mask of the on-site orbital matrix
    unsigned soz_nz[6];     // per row: bit 2*b2 real part, bit 2*b2+1 imaginary part
    unsigned pair_phase;    // bit d: pair d carries a Peierls phase
};

// Peierls phase storage:
//  PH_NONE: B = 0
//  PH_SYM:  symmetric gauge; theta(r, r+delta) = -theta(r, r-delta) = phi_d(r),
//           table [Np][9] of (cos phi_d, sin phi_d)
//  PH_GEN:  any gauge; table [Np][18] of exp(-i theta) per link (+delta, -delta)
enum { PH_NONE = 0, PH_SYM = 1, PH_GEN = 2 };

template <typename R>
struct StencilArgs {
    int nx, ny, nz;
    int ld;             // complex elements per row of x, prev, y
    int col0, ncol;     // processed columns
    R alpha, beta, gamma;   // y = alpha*H x + beta*x + gamma*prev
    const cx_t<R>* x;
    const cx_t<R>* prev;    // may be null when gamma == 0
    cx_t<R>* y;
    const R* onsite;        // [Np][6] on-site orbital matrix (centre + V + strain)
    const cx_t<R>* phase;   // see PH_*; null when B = 0
    int phase_mode;
    const uint8_t* mask;    // [Np] or null
    // optional source term: y += src_coef[col] * src (defect-corrected filter)
    const cx_t<R>* src;     // same layout as y, or null
    R src_coef[64];
    Coeffs<R> c;
    int nb;                 // bands per point: 6, or 3 for the spin-independent H0
    int* err;               // device status word (bit 8: a pipeline wait ran out), or null
};

}  // namespace khp

// ------------------------------------------------------------------ handle
struct khp_grid {
    int nx, ny, nz;
    int nb;                // bands per point: 6 (k.p with spin-orbit) or 3 (spin-independent H0)
    long long np;          // points
    long long n;           // unknowns = nb np
    double h;
    khp_material mat;
    double rot[9];
    cudaStream_t stream;
    int device;

    // host copies of the constant operator pieces (FP64)
    double hop[9][6];
    double center[6];
    double soz_re[6][6], soz_im[6][6];
    double De[6][6];       // dH'_PB/deps_c per strain component c, sym 3x3
    double B[3];
    int gauge;
    bool fields_set;
    bool has_phase;
    bool has_strain;
    int phase_mode;        // PH_NONE / PH_SYM / PH_GEN
    unsigned pair_phase;   // pairs with a nonzero phase
    double onsite_absmax;  // max over points of the on-site orbital row sums

    // device fields
    uint8_t* mask;         // [np] or null
    double* onsite64;      // [np][6]
    float* onsite32;       // [np][6]
    double2* phase64;      // [np][18] or null
    float2* phase32;       // [np][18] or null

    // workspace (grown on demand)
    int ws_m;
    double2* blk64[4];     // FP64 blocks [n][ws_m]
    float2* blk32[4];      // FP32 blocks [n][ws_m]
    int ws_has32;
    double2* partial;      // reduction partials
    size_t partial_elems;
    double2* small;        // m x m matrices on device (G, S, Q, Rinv ...)
    double* dvec;          // device vectors (theta, residuals, misc)
    int* dflag;            // device status flags
    double* host_pinned;   // pinned host staging

    double* lz;            // Lanczos scratch: partials, alpha, beta
    bool bound_valid;      // lambda_lanczos matches the current fields
    double lambda_lanczos; // Lanczos upper bound of the spectrum
    double lambda_low;     // Lanczos lower estimate of the spectrum

    double ctr[3];         // symmetric-gauge centre when ctr_set (else the box centre)
    int ctr_set;
    khp_grid* coarse;      // coarse-grid start: the handle of the 2x coarser grid, or null
    double2* coarse_x;     // its start block [n_coarse][coarse_m]
    int coarse_m;
    bool coarse_valid;     // coarse fields match the current fine fields

    long long launches;    // kernel launches issued (per call accounting)
    cudaEvent_t ev0, ev1;  // filter timing
    cudaEvent_t evp[5];    // phase timing: Gram | small problem | rotation, and the H Y apply
};
