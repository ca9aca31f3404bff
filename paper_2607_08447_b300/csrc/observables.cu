// Hole density and Hellmann-Feynman adjoint of the lowest eigenpairs.
//   rho(p)       = sum_i w_i sum_b |psi_i(6p+b)|^2             (Sec. II B)
//   dL/dV(p)     = sum_i g_i sum_b |psi_i(6p+b)|^2             (dH/dV(p) = 1 at p)
//   dL/deps_c(p) = sum_i g_i sum_s psi_i(p,s)^H M_c psi_i(p,s) (M_c = dH'_PB/deps_c)
//   dL/dalpha_g  = sum_p dL/dV(p) Phi_g(p)
// Every sum runs in a fixed order (states outer, bands inner; points in
// block order), so results are bitwise reproducible.
#include "khp_common.cuh"
#include "khp_internal.h"

namespace khp {

struct DensityArgs {
    const double2* psi;
    long long np;
    int n;
    int nb;                // bands per point (6, or 3 for the spin-independent H0)
    double w[KHP_MAX_M];
    double* rho;
};

__global__ void density_kernel(const DensityArgs a) {
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= a.np) return;
    const double2* row = a.psi + p * a.nb * a.n;
    double rho = 0.0;
    for (int i = 0; i < a.n; ++i) {
        double s = 0.0;
        for (int b = 0; b < a.nb; ++b) {
            const double2 v = row[b * a.n + i];
            s += v.x * v.x + v.y * v.y;
        }
        rho += a.w[i] * s;
    }
    a.rho[p] = rho;
}

cudaError_t launch_density(const double2* psi, long long np, int n, const double* w,
                           const uint8_t* /*mask*/, double* rho, cudaStream_t st, int nb) {
    DensityArgs a;
    a.psi = psi; a.np = np; a.n = n; a.nb = nb; a.rho = rho;
    for (int i = 0; i < KHP_MAX_M; ++i) a.w[i] = i < n ? w[i] : 0.0;
    density_kernel<<<(unsigned)((np + 255) / 256), 256, 0, st>>>(a);
    return cudaGetLastError();
}

struct BackArgs {
    const double2* psi;
    long long np;
    int n;
    int nb;                // bands per point (6, or 3 for the spin-independent H0)
    double g[KHP_MAX_M];
    double De[6][6];       // sym 3x3 (00,11,22,12,02,01) per strain component
    double* dV;
    double* dEps;          // [6][np] or null
    const double* levers;  // [ng][np] or null
    int ng;
    double* partial;       // [gridDim][ng]
};

__device__ __forceinline__ double quad_sym(const double* M, const double2 x0, const double2 x1,
                                           const double2 x2) {
    // Re(x^H M x) for real symmetric M
    const double d = M[0] * (x0.x * x0.x + x0.y * x0.y) + M[1] * (x1.x * x1.x + x1.y * x1.y) +
                     M[2] * (x2.x * x2.x + x2.y * x2.y);
    const double o = M[3] * (x1.x * x2.x + x1.y * x2.y) + M[4] * (x0.x * x2.x + x0.y * x2.y) +
                     M[5] * (x0.x * x1.x + x0.y * x1.y);
    return d + 2.0 * o;
}

__global__ void backward_kernel(const BackArgs a) {
    __shared__ double red[256];
    const long long per = (a.np + gridDim.x - 1) / gridDim.x;
    const long long p0 = (long long)blockIdx.x * per;
    const long long p1 = p0 + per < a.np ? p0 + per : a.np;
    double lev[KHP_MAX_GATES];
    for (int g = 0; g < KHP_MAX_GATES; ++g) lev[g] = 0.0;
    for (long long p = p0 + threadIdx.x; p < p1; p += blockDim.x) {
        const double2* row = a.psi + p * a.nb * a.n;
        double dv = 0.0;
        double de[6] = {0, 0, 0, 0, 0, 0};
        const bool two = a.nb == 6;
        for (int i = 0; i < a.n; ++i) {
            double2 x[6];
#pragma unroll
            for (int b = 0; b < 6; ++b) x[b] = (b < 3 || two) ? row[b * a.n + i] : make_double2(0.0, 0.0);
            double s = 0.0;
#pragma unroll
            for (int b = 0; b < 6; ++b) s += x[b].x * x[b].x + x[b].y * x[b].y;
            dv += a.g[i] * s;
            if (a.dEps) {
#pragma unroll
                for (int c = 0; c < 6; ++c)
                    de[c] += a.g[i] * (quad_sym(a.De[c], x[0], x[1], x[2]) + quad_sym(a.De[c], x[3], x[4], x[5]));
            }
        }
        a.dV[p] = dv;
        if (a.dEps)
            for (int c = 0; c < 6; ++c) a.dEps[(long long)c * a.np + p] = de[c];
        for (int g = 0; g < a.ng; ++g) lev[g] += dv * a.levers[(long long)g * a.np + p];
    }
    for (int g = 0; g < a.ng; ++g) {
        red[threadIdx.x] = lev[g];
        __syncthreads();
        for (int s = blockDim.x / 2; s > 0; s >>= 1) {
            if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
            __syncthreads();
        }
        if (threadIdx.x == 0) a.partial[(size_t)blockIdx.x * a.ng + g] = red[0];
        __syncthreads();
    }
}

__global__ void lever_finish(const double* partial, int nblk, int ng, double* out) {
    const int g = threadIdx.x;
    if (g >= ng) return;
    double s = 0.0;
    for (int b = 0; b < nblk; ++b) s += partial[(size_t)b * ng + g];
    out[g] = s;
}

cudaError_t launch_backward(const double2* psi, long long np, int n, const double* g,
                            const double (*De)[6], double* dV, double* dEps, const double* levers,
                            int ng, double* partial, int nblk, double* dalpha_dev, cudaStream_t st, int nb) {
    BackArgs a;
    a.psi = psi; a.np = np; a.n = n; a.nb = nb;
    for (int i = 0; i < KHP_MAX_M; ++i) a.g[i] = i < n ? g[i] : 0.0;
    for (int c = 0; c < 6; ++c)
        for (int k = 0; k < 6; ++k) a.De[c][k] = De[c][k];
    a.dV = dV; a.dEps = dEps; a.levers = levers; a.ng = levers ? ng : 0; a.partial = partial;
    backward_kernel<<<nblk, 256, 0, st>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || a.ng == 0) return e;
    lever_finish<<<1, 32, 0, st>>>(partial, nblk, a.ng, dalpha_dev);
    return cudaGetLastError();
}

}  // namespace khp

// ---------------------------------------------------------- pair densities
// rho_jl(p) = sum_b conj(psi_j(p, b)) psi_l(p, b) for every ordered pair
// (j, l) (the overlap densities of the Coulomb integrals of the CI step,
// Sec. II C, Eqs. 13-15), written as [Np][n * n] complex, pair index j n + l.
namespace khp {

// dens[i][p] = sum_b |psi_i(nb p + b)|^2: the per-state densities (discrete
// norm) of n states, state-major so that a state's density is contiguous
__global__ void state_density_kernel(const double2* __restrict__ psi, long long np, int n, int nb,
                                     double* __restrict__ dens) {
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= np) return;
    const double2* row = psi + p * nb * n;
    for (int i = 0; i < n; ++i) {
        double s = 0.0;
        for (int b = 0; b < nb; ++b) {
            const double2 v = row[b * n + i];
            s = fma(v.x, v.x, fma(v.y, v.y, s));
        }
        dens[(long long)i * np + p] = s;
    }
}

cudaError_t launch_state_densities(const double2* psi, long long np, int n, int nb, double* dens, cudaStream_t st) {
    state_density_kernel<<<(unsigned)((np + 255) / 256), 256, 0, st>>>(psi, np, n, nb, dens);
    return cudaGetLastError();
}

__global__ void pair_density_kernel(const double2* __restrict__ psi, long long np, int n, int nb,
                                    double2* __restrict__ out) {
    const int npair = n * n;
    const long long total = np * npair;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const long long p = t / npair;
        const int k = (int)(t - p * npair);
        const int j = k / n, l = k - j * n;
        const double2* row = psi + p * nb * n;
        double2 s = make_double2(0.0, 0.0);
        for (int b = 0; b < nb; ++b) cfmac(s, row[b * n + j], row[b * n + l]);
        out[t] = s;
    }
}

cudaError_t launch_pair_density(const double2* psi, long long np, int n, int nb, double2* out, cudaStream_t st) {
    const long long total = np * (long long)(n * n);
    long long blocks = (total + 255) / 256;
    if (blocks > 148 * 32) blocks = 148 * 32;
    if (blocks < 1) blocks = 1;
    pair_density_kernel<<<(unsigned)blocks, 256, 0, st>>>(psi, np, n, nb, out);
    return cudaGetLastError();
}

}  // namespace khp

// ------------------------------------------------------------------------
// First moments of a block of states about the box centre: the position
// operator projected on the states,
//   D_a[i][j] = sum_p r_a(p) sum_b conj(X_i(p, b)) X_j(p, b),
//   r_a(p) = (i_a(p) - (n_a - 1) / 2) h,   a = x, y, z,
// whose eigenvectors along the dot axis localise the bonding and
// anti-bonding doublets of a double dot on the left and right dots
// (g-tensors of Sec. III B).  One thread per packed pair (i <= j) and point
// group; a block sums its groups in group order, the blocks are summed in
// block order (sum_partials_herm), so the result is bitwise reproducible.
namespace khp {

__global__ void __launch_bounds__(256) moments_kernel(const double2* __restrict__ X, int nx, int ny,
                                                      long long np, int nb, int m, double h, double cx,
                                                      double cy, double cz, double2* __restrict__ partial) {
    extern __shared__ double2 acc_s[];   // [groups][3 mt]
    const int mt = m * (m + 1) / 2;
    const int groups = blockDim.x / mt;
    const int gi = threadIdx.x / mt;
    const int k = threadIdx.x - gi * mt;
    if (gi < groups) {
        int i, j;
        packed_ij(k, m, i, j);
        double2 ax = make_double2(0.0, 0.0), ay = ax, az = ax;
        for (long long p = (long long)blockIdx.x * groups + gi; p < np; p += (long long)gridDim.x * groups) {
            const double2* row = X + p * nb * m;
            double2 q = make_double2(0.0, 0.0);
            for (int b = 0; b < nb; ++b) cfmac(q, row[b * m + i], row[b * m + j]);
            const long long yz = p / nx;
            const double x = ((double)(p - yz * nx) - cx) * h;
            const double y = ((double)(yz % ny) - cy) * h;
            const double z = ((double)(yz / ny) - cz) * h;
            ax.x = fma(x, q.x, ax.x); ax.y = fma(x, q.y, ax.y);
            ay.x = fma(y, q.x, ay.x); ay.y = fma(y, q.y, ay.y);
            az.x = fma(z, q.x, az.x); az.y = fma(z, q.y, az.y);
        }
        double2* a = acc_s + gi * 3 * mt;
        a[k] = ax;
        a[mt + k] = ay;
        a[2 * mt + k] = az;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < 3 * mt; e += blockDim.x) {
        double2 s = make_double2(0.0, 0.0);
        for (int g = 0; g < groups; ++g) {
            const double2 v = acc_s[g * 3 * mt + e];
            s.x += v.x;
            s.y += v.y;
        }
        partial[(size_t)blockIdx.x * 3 * mt + e] = s;
    }
}

cudaError_t launch_moments(const double2* X, int nx, int ny, int nz, int nb, int m, double h, double2* partial,
                           size_t partial_elems, double2* out, cudaStream_t st) {
    const int mt = m * (m + 1) / 2;
    const int groups = 256 / mt;
    const long long np = (long long)nx * ny * nz;
    long long blocks = (np + groups - 1) / groups;
    blocks = std::min<long long>(blocks, 148 * 4);
    blocks = std::min<long long>(blocks, (long long)(partial_elems / (3 * mt)));
    if (blocks < 1) return cudaErrorInvalidValue;
    const size_t smem = sizeof(double2) * groups * 3 * mt;
    moments_kernel<<<(unsigned)blocks, 256, smem, st>>>(X, nx, ny, np, nb, m, h, 0.5 * (nx - 1),
                                                       0.5 * (ny - 1), 0.5 * (nz - 1), partial);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_sum_partials_herm(partial, (int)blocks, m, 3, out, st);
}

}  // namespace khp
