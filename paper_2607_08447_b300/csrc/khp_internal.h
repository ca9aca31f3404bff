// Internal launchers and constants shared by the library's translation units.
#pragma once

#include <string>

#include "khp_common.cuh"

#define KHP_MAX_GATES 16
#define KHP_MAX_M 64
#define KHP_MAX_MOMENT_M 16
#define KHP_PHI0 658.2119569        /* hbar / e  [T nm^2] */
#define KHP_MU_B 5.7883818060e-5    /* Bohr magneton [eV / T] */
#define KHP_HB2M 0.0380998212       /* hbar^2 / (2 m0) [eV nm^2] */

namespace khp {

// stencil.cu
template <typename R>
cudaError_t launch_stencil(const StencilArgs<R>& a, cudaStream_t st);
// plane-marching FP32 stencil (TMA-staged planes); cudaErrorNotSupported
// when the step is outside what it covers (the caller then uses the
// per-point kernel).  prepare_plane() opts its kernels into their shared
// memory (per device, outside stream capture).
cudaError_t launch_stencil_plane(const StencilArgs<float>& a, int* err, cudaStream_t st);
// the same step of `count` problems in grouped launches (batched rounds);
// cudaErrorNotSupported, with nothing launched, when the plane kernel does
// not cover all of them alike
cudaError_t launch_stencil_plane_group(const StencilArgs<float>* const* a, int count, cudaStream_t st);
cudaError_t prepare_plane();
cudaError_t launch_field_setup(khp_grid* g, const double* V, const double* strain,
                               const double* levers, const double* alpha, int ng, int* bad);
cudaError_t launch_phase_setup(khp_grid* g);
cudaError_t launch_onsite_rowmax(khp_grid* g, double* partial, int nblocks, double* out);

// coarse.cu: the coarse-grid start.  The coarse grid takes every second
// point (fine index 2j + 1, 0-based) at twice the spacing; its on-site
// block is the fine one at those points with the fine kinetic diagonal
// replaced by the coarse one.  The prolongation fills the fine block by
// trilinear interpolation (zero at the walls and at masked points).
cudaError_t launch_restrict_onsite(const khp_grid* fine, khp_grid* coarse);
cudaError_t launch_prolong(const khp_grid* coarse, const double2* Xc, int ldc, const khp_grid* fine, double2* X,
                           int ld, int ncol);

// dense.cu
int dense_blocks(long long rows);
size_t gram_partial_elems(int m, int nblk);
// partial[nblk][2 m m]; out[0 .. m*m) = Y^H Y, out[m*m .. 2 m*m) = Y^H W (if W)
cudaError_t launch_gram(const double2* Y, const double2* W, long long rows, int ld, int col0,
                        int m, double2* partial, int nblk, double2* out, cudaStream_t st);
// X[:, col0_out + j] = sum_i Y[:, col0_in + i] Q[i][j] (and HX from W), j < mq;
// optional residual norms ||HX_j - theta_j X_j|| / ||X_j|| into res_out[mq]
cudaError_t launch_rotate(const double2* Y, const double2* W, int ld, int col0, int m,
                          const double2* Q, int mq, const double* theta, double2* X, double2* HX,
                          long long rows, double* res_partial, int nblk, double* res_out,
                          cudaStream_t st);
// reducers shared with the tensor-core projections
cudaError_t launch_sum_partials_herm(const double2* partial, int nblk, int m, int nmat, double2* out,
                                     cudaStream_t st);
cudaError_t launch_residual_finish(const double* partial, int nblk, int mq, double* out, cudaStream_t st);

// ozaki.cu: the same Gram and rotation contractions (same arguments and
// outputs) as exact split-digit BF16 products on the tensor cores, FP64
// accurate; m, mq <= 32 (oz_supported).  prepare_oz() opts the kernels into
// their shared memory (per device, outside stream capture).
bool oz_supported(int m, int mq);
cudaError_t prepare_oz();
cudaError_t launch_gram_oz(const double2* Y, const double2* W, long long rows, int ld, int col0, int m,
                           double2* partial, int nblk, double2* out, cudaStream_t st);
cudaError_t launch_rotate_oz(const double2* Y, const double2* W, int ld, int col0, int m, const double2* Q,
                             int mq, const double* theta, double2* X, double2* HX, long long rows,
                             double* res_partial, int nblk, double* res_out, cudaStream_t st);

// ozaki_tc.cu: the same contractions and outputs with the digit products on
// the 5th-generation tensor cores (tcgen05.mma, accumulators in TMEM); m, mq
// <= 32 (tc_supported).  A bounded wait that runs out sets bit 8 of *err.
// prepare_tc() opts the kernels into their shared memory.
bool tc_supported(int m, int mq);
cudaError_t prepare_tc();
cudaError_t launch_gram_tc(const double2* Y, const double2* W, long long rows, int ld, int col0, int m,
                           double2* partial, int nblk, double2* out, int* err, cudaStream_t st);
cudaError_t launch_rotate_tc(const double2* Y, const double2* W, int ld, int col0, int m, const double2* Q,
                             int mq, const double* theta, double2* X, double2* HX, long long rows,
                             double* res_partial, int nblk, double* res_out, int* err, cudaStream_t st);

// mode 0: Q = R^-1 of the (equilibrated) Cholesky factor of G (G = R^H R)
// mode 1: generalized Rayleigh-Ritz  S q = theta G q  ->  theta ascending,
//         Q = R^-1 Qhat (columns G-orthonormal)
// flags[0] |= 1 shifted Cholesky, 2 breakdown, 4 non-finite
cudaError_t launch_small(const double2* G, const double2* S, int m, int mode, double2* Q,
                         double* theta, int* flags, cudaStream_t st);
cudaError_t launch_convert_d2f(const double2* src, float2* dst, long long rows, int ld, int col0, int ncol,
                               cudaStream_t st);
cudaError_t launch_convert_f2d(const float2* src, double2* dst, long long rows, int ld, int col0, int ncol,
                               cudaStream_t st);
cudaError_t launch_random_fill(double2* X, long long rows, int ld, int col0, int ncol,
                               unsigned long long seed, const uint8_t* mask, cudaStream_t st, int bands = 6);

// Lanczos pieces (dense.cu); scalars live in device memory
cudaError_t lanczos_dot(const double2* a, const double2* b, long long n, double* partial, double* out,
                        cudaStream_t st);
cudaError_t lanczos_orth(double2* w, const double2* v, const double2* vprev, const double* alpha,
                         const double* beta_prev, double* beta_out, long long n, double* partial,
                         cudaStream_t st);
cudaError_t lanczos_norm(const double2* v, long long n, double* partial, double* out, cudaStream_t st);
cudaError_t lanczos_scale(double2* dst, const double2* src, const double* nrm, long long n, cudaStream_t st);
cudaError_t lanczos_tridiag(const double* alpha, const double* beta, int k, double2* G, double2* S,
                            cudaStream_t st);

// defect-corrected FP32 filter (dense.cu)
cudaError_t launch_dc_residual(const double2* X, const double2* HX, float2* R, float2* Z1, long long rows,
                               int ld, int col0, int ncol, const double* theta, double alpha0,
                               cudaStream_t st);
cudaError_t launch_dc_combine(const double2* X, const double2* HX, const float2* Z, double2* Y, double2* W,
                              long long rows, int ld, int zcol0, const double* D, cudaStream_t st);

// observables.cu
cudaError_t launch_state_densities(const double2* psi, long long np, int n, int nb, double* dens, cudaStream_t st);
cudaError_t launch_pair_density(const double2* psi, long long np, int n, int nb, double2* out, cudaStream_t st);
// D [3][m][m] = first moments of the m states X about the box centre
// (partial: scratch of partial_elems entries)
cudaError_t launch_moments(const double2* X, int nx, int ny, int nz, int nb, int m, double h, double2* partial,
                           size_t partial_elems, double2* out, cudaStream_t st);
cudaError_t launch_density(const double2* psi, long long np, int n, const double* w,
                           const uint8_t* mask, double* rho, cudaStream_t st, int nb = 6);
cudaError_t launch_backward(const double2* psi, long long np, int n, const double* g,
                            const double (*De)[6], double* dV, double* dEps,
                            const double* levers, int ng, double* partial, int nblk,
                            double* dalpha_dev, cudaStream_t st, int nb = 6);

}  // namespace khp

// Records the message returned by khp_last_error() on this thread and
// passes the status through (khp_api.cu).
khp_status khp_set_error(khp_status s, const std::string& msg);
// Clears the calling thread's last-error message (start of every entry point).
void khp_clear_error();
