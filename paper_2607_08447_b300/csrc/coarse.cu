// Coarse-grid start of the eigensolve: the on-site fields restricted to the
// grid of every second point at twice the spacing, and the trilinear
// prolongation of a coarse block back to the fine grid.
//
// Geometry: with Dirichlet walls at 0 and (n + 1) h, fine point i (0-based)
// sits at (i + 1) h and coarse point j at (j + 1) 2h = fine point 2j + 1.
// A fine point with odd i coincides with coarse point (i - 1) / 2; one with
// even i lies halfway between coarse points i/2 - 1 and i/2 (a wall, value
// zero, where either is outside the coarse grid).
#include "khp_common.cuh"
#include "khp_internal.h"

namespace khp {
namespace {

struct RestrictArgs {
    int nxc, nyc, nzc, nx, ny;
    double dcent[6];          // coarse minus fine kinetic diagonal of the on-site block
    const double* on64;       // fine [np][6]
    double* oc64;             // coarse [npc][6]
    float* oc32;
    const uint8_t* mask;      // fine mask or null
    uint8_t* maskc;           // coarse mask or null
};

__global__ void restrict_kernel(const RestrictArgs a) {
    const long long npc = (long long)a.nxc * a.nyc * a.nzc;
    const long long pc = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (pc >= npc) return;
    const int jx = (int)(pc % a.nxc);
    const long long q = pc / a.nxc;
    const int jy = (int)(q % a.nyc);
    const int jz = (int)(q / a.nyc);
    const long long pf = (2LL * jx + 1) + (long long)a.nx * ((2LL * jy + 1) + (long long)a.ny * (2LL * jz + 1));
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        const double v = a.on64[pf * 6 + k] + a.dcent[k];
        a.oc64[pc * 6 + k] = v;
        a.oc32[pc * 6 + k] = (float)v;
    }
    if (a.maskc) a.maskc[pc] = a.mask[pf];
}

// coarse neighbours of fine index i along one axis (nc coarse points)
__device__ __forceinline__ int axis_weights(int i, int nc, int (&j)[2], double (&w)[2]) {
    if (i & 1) {
        j[0] = (i - 1) >> 1;
        w[0] = 1.0;
        return 1;
    }
    int n = 0;
    const int jl = (i >> 1) - 1, jh = i >> 1;
    if (jl >= 0) { j[n] = jl; w[n] = 0.5; ++n; }
    if (jh < nc) { j[n] = jh; w[n] = 0.5; ++n; }
    return n;
}

struct ProlongArgs {
    int nx, ny, nz, nxc, nyc, nzc, nb, ldc, ld, ncol;
    const double2* Xc;        // coarse [npc nb][ldc]
    double2* X;               // fine [np nb][ld]
    const uint8_t* mask;      // fine mask or null
};

// one thread per (fine point, band, column)
__global__ void prolong_kernel(const ProlongArgs a) {
    const long long np = (long long)a.nx * a.ny * a.nz;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= np * a.nb * a.ncol) return;
    const int c = (int)(t % a.ncol);
    const long long r = t / a.ncol;
    const int b = (int)(r % a.nb);
    const long long p = r / a.nb;
    double2 s = make_double2(0.0, 0.0);
    if (!a.mask || a.mask[p]) {
        const int ix = (int)(p % a.nx);
        const long long q = p / a.nx;
        const int iy = (int)(q % a.ny);
        const int iz = (int)(q / a.ny);
        int jx[2], jy[2], jz[2];
        double wx[2], wy[2], wz[2];
        const int nxw = axis_weights(ix, a.nxc, jx, wx);
        const int nyw = axis_weights(iy, a.nyc, jy, wy);
        const int nzw = axis_weights(iz, a.nzc, jz, wz);
        for (int u = 0; u < nzw; ++u)
            for (int v = 0; v < nyw; ++v)
                for (int x = 0; x < nxw; ++x) {
                    const double w = wz[u] * wy[v] * wx[x];
                    const long long pc = jx[x] + (long long)a.nxc * (jy[v] + (long long)a.nyc * jz[u]);
                    const double2 y = a.Xc[(pc * a.nb + b) * a.ldc + c];
                    s.x = fma(w, y.x, s.x);
                    s.y = fma(w, y.y, s.y);
                }
    }
    a.X[(p * a.nb + b) * a.ld + c] = s;
}

}  // namespace

cudaError_t launch_restrict_onsite(const khp_grid* fine, khp_grid* coarse) {
    RestrictArgs a;
    a.nxc = coarse->nx; a.nyc = coarse->ny; a.nzc = coarse->nz;
    a.nx = fine->nx; a.ny = fine->ny;
    for (int k = 0; k < 6; ++k) a.dcent[k] = coarse->center[k] - fine->center[k];
    a.on64 = fine->onsite64;
    a.oc64 = coarse->onsite64;
    a.oc32 = coarse->onsite32;
    a.mask = fine->mask;
    a.maskc = fine->mask ? coarse->mask : nullptr;
    const int threads = 256;
    const long long blocks = (coarse->np + threads - 1) / threads;
    restrict_kernel<<<(unsigned)blocks, threads, 0, fine->stream>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_prolong(const khp_grid* coarse, const double2* Xc, int ldc, const khp_grid* fine, double2* X,
                           int ld, int ncol) {
    ProlongArgs a;
    a.nx = fine->nx; a.ny = fine->ny; a.nz = fine->nz;
    a.nxc = coarse->nx; a.nyc = coarse->ny; a.nzc = coarse->nz;
    a.nb = fine->nb; a.ldc = ldc; a.ld = ld; a.ncol = ncol;
    a.Xc = Xc; a.X = X; a.mask = fine->mask;
    const int threads = 256;
    const long long total = fine->np * fine->nb * ncol;
    const long long blocks = (total + threads - 1) / threads;
    prolong_kernel<<<(unsigned)blocks, threads, 0, fine->stream>>>(a);
    return cudaGetLastError();
}

}  // namespace khp
