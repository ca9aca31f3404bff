/*
 * khp.h -- C ABI of the B300 k.p hole eigensolver.
 *
 * The library computes the lowest confined hole states of the discretised
 * 6x6 Luttinger-Kohn k.p Hamiltonian with Bir-Pikus strain and a magnetic
 * field, H_NI = H_LK + H_PB + V (paper Eq. 2b), written in the
 * |X,Y,Z> x {up,down} basis as H_DKK + H_SOI + H'_PB + V (Eqs. 5-6a), on a
 * uniform finite-difference grid with Dirichlet walls (Sec. II B), by
 * Chebyshev-filtered subspace iteration (the Rayleigh-Chebyshev method named
 * in Sec. II B).  All arithmetic runs in the library's CUDA kernels.
 *
 * Conventions (every entry point):
 *  - grid: nx*ny*nz interior points, spacing h [nm]; point (ix,iy,iz) sits at
 *    ((ix+1)h, (iy+1)h, (iz+1)h); the wave function vanishes outside.
 *    Point index p = ix + nx*(iy + ny*iz).  N = 6*nx*ny*nz unknowns.
 *  - unknown index (row) = 6*p + b with b = 3*s + o, o in {X,Y,Z} (grid
 *    frame), s in {up, down} (spin quantised along grid z).
 *  - blocks of vectors are ROW-MAJOR [N][m] arrays of interleaved complex
 *    numbers (complex128 = 2 doubles, or complex64 = 2 floats where stated):
 *    element (row, j) at offset row*m + j.  Column j is vector j.
 *  - energies eV, lengths nm, magnetic field tesla.
 *  - "_dev" pointers are device pointers of the current CUDA device, "_host"
 *    pointers are host memory.  The caller owns every buffer it passes; the
 *    library owns only the handle and its workspace.  Nothing crosses the
 *    boundary with ownership.
 *  - every call returns a khp_status; nothing aborts.  On error the handle
 *    is left usable and khp_last_error() describes the failure.
 *  - all device work of a handle is issued on the stream given at creation;
 *    calls that return host results synchronise that stream.
 */
#ifndef KHP_H
#define KHP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define KHP_STATS_HISTORY 64

typedef struct khp_grid* khp_handle;

typedef enum {
    KHP_OK = 0,
    KHP_ERR_INVALID_ARG = 1,   /* bad size, null pointer, NaN input ...       */
    KHP_ERR_CUDA = 2,          /* a CUDA runtime call failed                    */
    KHP_ERR_OOM = 3,           /* device allocation of the workspace failed     */
    KHP_ERR_NOT_CONVERGED = 4, /* max_iter reached; results hold current Ritz pairs */
    KHP_ERR_BREAKDOWN = 5,     /* Cholesky of the Gram matrix failed even shifted */
    KHP_ERR_STATE = 6,         /* call out of order (e.g. solve before fields)  */
    KHP_ERR_DEGENERATE = 7     /* gradient asked for a split degenerate cluster */
} khp_status;

/* Material parameters (Table I of the paper has one Si set): Luttinger
 * gamma1..3, split-off energy delta_so [eV], isotropic magnetic kappa,
 * deformation potentials a_v, b, d [eV]. */
typedef struct {
    double gamma1, gamma2, gamma3, delta_so, kappa, a_v, b, d;
} khp_material;

/* Eigensolver options.
 *  n_states       wanted lowest states (1..block_m-1)
 *  block_m        subspace width, even, n_states < block_m <= 64
 *  degree         Chebyshev filter degree per outer iteration (>= 1)
 *  max_iter       outer-iteration cap
 *  precision      0: plain FP64 throughout;
 *                 1: mixed: FP32 Chebyshev filter/stencil with FP64
 *                    Cholesky and Rayleigh-Ritz until the FP32 residual
 *                    floor, then FP64 refinement sweeps (wide-window FP64
 *                    clean-up sweeps, then FP64 filter + Rayleigh-Ritz);
 *                 2: defect-corrected FP32: the filtered block is written as
 *                    Y = X p(Theta) + Z with p(Theta) the FP64 scalar
 *                    recurrence at the Ritz values and Z driven by the FP64
 *                    residual H X - X Theta; every filter apply runs in FP32
 *                    on Z, H Y in FP64 and an FP64-accurate Rayleigh-Ritz
 *                    (see projections).  Reaches the
 *                    plain-FP64 accuracy (tested to 1e-10 eV).
 *  refine_sweeps  precision 1 only: number of FP64 clean-up sweeps; < 0 means
 *                 one clean-up sweep, then FP64 sweeps until every residual is
 *                 below tol_ev
 *  tol_ev         stop when ||H x_i - theta_i x_i|| <= tol_ev for i < n_states
 *  seed           seed of the counter-based random start vectors
 *  warm_start_dev optional complex128 [N][warm_cols] start vectors (row-major);
 *                 remaining columns are random.  NULL for a cold start.
 *  projections    how the Rayleigh-Ritz contractions (Gram matrices and
 *                 subspace rotation) run: 0 = on the 5th-generation tensor
 *                 cores (tcgen05.mma, accumulators in TMEM) as exact
 *                 split-digit BF16 products recombined in FP64 (FP64
 *                 accurate; block_m <= 32, wider blocks use 1); 1 = FP64
 *                 ALU; 2 = the same split-digit products through the
 *                 warp-level mma.sync path.  Zero-initialised options
 *                 select 0.
 *  start          start block when warm_start_dev is NULL: 0 = random
 *                 (counter-based, from seed); 1 = coarse grid: the lowest
 *                 block_m states of the grid of every second point at twice
 *                 the spacing (on-site fields restricted, same material,
 *                 field and gauge), solved loosely (tolerance max(tol_ev,
 *                 1e-3) eV, degree 120 plain / 60 otherwise, block_m + 8
 *                 columns; KHP_COARSE="degree,tol,extra" in the environment
 *                 replaces these) and prolongated trilinearly; falls
 *                 back to 0 when that grid has fewer than 4 (block_m + 8)
 *                 unknowns or block_m + 8 > 64.  khp_eigensolve only.
 *  block_out_dev  optional complex128 [N][block_m] output (row-major): the
 *                 final orthonormal Ritz block, all block_m columns (the
 *                 n_states eigenvectors first, then the guard columns), a
 *                 start block for a solve of a nearby Hamiltonian through
 *                 warm_start_dev.  NULL: not written.  khp_eigensolve only. */
typedef struct {
    int n_states;
    int block_m;
    int degree;
    int max_iter;
    int precision;
    int refine_sweeps;
    double tol_ev;
    uint64_t seed;
    const void* warm_start_dev;
    int warm_cols;
    int projections;
    int start;
    void* block_out_dev;
} khp_solver_opts;

/* Per-solve statistics (optional output).  The filter timings come from
 * CUDA events recorded on the handle's stream around each Chebyshev filter
 * (the fused stencil launches only); the algorithmic counts describe one
 * application of H to one vector at one interior grid point. */
typedef struct {
    int iterations;            /* outer iterations done (all precisions)       */
    int iterations_fp32;       /* of which with the FP32 filter                */
    int converged;             /* states with residual <= tol_ev               */
    int shifted_cholesky;      /* times the Gram Cholesky needed a shift        */
    long long filter_applies;  /* block stencil applications (any precision)   */
    double max_residual;       /* max over the n_states residual norms [eV]    */
    double lambda_upper;       /* upper spectral bound used by the filter [eV] */
    double ms_total;           /* wall time of the call [ms]                    */
    double ms_filter_fp64;     /* device time of the FP64 filters [ms]          */
    double ms_filter_fp32;     /* device time of the FP32 filters [ms]          */
    long long launches_fp64;   /* fused stencil launches inside FP64 filters    */
    long long launches_fp32;   /* fused stencil launches inside FP32 filters    */
    long long kernel_launches; /* all library kernel launches of the call       */
    double point_vectors;      /* grid points x block width of one launch      */
    double pv_fp64;            /* point-vectors processed by the FP64 filters   */
    double pv_fp32;            /* point-vectors processed by the FP32 filters   */
    double flops_per_pv;       /* sparse H x (8 flop per complex, 4 per real
                                  nonzero) + the three-term update, per point-vector */
    double bytes_per_pv_fp64;  /* algorithmic HBM bytes per point-vector of a
                                  filter step: read Y_k, Y_k-1, write Y_k+1 and
                                  the per-point field tables over the block width */
    double bytes_per_pv_fp32;
    int block_m;               /* block width used (after autotuning)          */
    int batch_rounds;          /* batched call: lock-step rounds executed      */
    int batch_graphs;          /* batched call: CUDA graphs instantiated       */
    double autotune_ms;        /* batched call: time spent in autotune trials  */
    /* per-phase device time (CUDA events on the handle's stream; single
     * solves only): Gram matrices G = Y^H Y, S = Y^H W; the m x m problem;
     * the rotation X = Y Q, HX = W Q with the residual norms; and the work
     * between the filter and the Gram (block combine and the H Y apply) */
    double ms_gram, ms_small, ms_rotate, ms_between;
    double bytes_rr;           /* algorithmic HBM bytes of the Gram and rotation passes */
    int n_history;             /* outer iterations recorded (incl. the start)  */
    double res_history[KHP_STATS_HISTORY]; /* max residual [eV] after each (first 64) */
    double ms_start;           /* wall time of the coarse-grid start [ms]      */
    int start_iterations;      /* outer iterations of the coarse-grid solve    */
} khp_stats;

/* Create a grid handle.
 *  rot     3x3 row-major; row a = grid axis a in crystal coordinates (an
 *          orthonormal matrix).  NULL = identity.  The paper's device frame
 *          (Sec. II A) is x=[110], y=[-110], z=[001].
 *  mask_dev optional uint8 [Np] device array, 0 = point excluded (Dirichlet
 *          there too).  NULL = every point active.  Copied at creation.
 *  stream  cudaStream_t (as void*) on which all work of this handle runs;
 *          NULL = the legacy default stream.
 * Errors: INVALID_ARG for non-positive sizes / h, non-orthonormal rot;
 *         OOM / CUDA on allocation failure. */
khp_status khp_create_grid(khp_handle* out, int nx, int ny, int nz, double h_nm,
                           const khp_material* mat, const double rot[9],
                           const uint8_t* mask_dev, void* stream);

/* Create a handle for the spin-independent single-particle Hamiltonian H0
 * (Sec. II C, Eq. 6a): without spin-orbit coupling the 6x6 Hamiltonian splits
 * into two identical 3x3 blocks (kinetic Luttinger term plus Bir-Pikus strain
 * plus V, on the orbitals X, Y, Z), and only one is kept.  Its eigenstates
 * form the orbital basis of the configuration-interaction step.
 * Same arguments and errors as khp_create_grid; delta_so and kappa of the
 * material are not used.  Every other entry point takes the handle with
 * N = 3 Np unknowns: row index 3 p + o, o = X, Y, Z.
 * khp_set_potential_strain_field rejects a nonzero B (INVALID_ARG): H0 has
 * no magnetic field. */
khp_status khp_create_grid_h0(khp_handle* out, int nx, int ny, int nz, double h_nm,
                              const khp_material* mat, const double rot[9], const uint8_t* mask_dev,
                              void* stream);

/* Set the fields of H (Eq. 2b: V_DQD and the strain entering H_PB; plus B).
 *  V_dev       float64 [Np] hole potential energy [eV], added as +V
 *  strain_dev  float64 [6][Np] strain tensor (xx,yy,zz,yz,xz,xy) in the grid
 *              frame, or NULL for no strain
 *  levers_dev  float64 [n_gates][Np] gate-lever fields Phi_g, or NULL; the
 *              potential used is V + sum_g alpha_host[g] * Phi_g
 *  alpha_host  float64 [n_gates] lever coefficients (NULL when n_gates = 0)
 *  B_host      3 doubles [T] in the grid frame (NULL = zero field)
 *  gauge       0 symmetric about the box centre, 1 Landau A=(0,Bz x-Bx z,-By x)
 * The arrays are read during the call (stream-ordered) and not retained.
 * Errors: INVALID_ARG for NULL V, bad gauge, n_gates < 0 or NaN/Inf in V. */
khp_status khp_set_potential_strain_field(khp_handle h, const double* V_dev,
                                          const double* strain_dev,
                                          const double* levers_dev,
                                          const double* alpha_host, int n_gates,
                                          const double* B_host, int gauge);

/* Y = H X for a block of m vectors (the matrix-free 19-point stencil).
 *  precision 0: X_dev, Y_dev complex128 [N][m];  1: complex64 [N][m].
 *  X and Y must not overlap.  m in 1..64 (m even for precision 1 fast path;
 *  odd m handled too). */
khp_status khp_apply(khp_handle h, const void* X_dev, void* Y_dev, int m, int precision);

/* One fused step of the Chebyshev filter (the three-term recurrence of the
 * Rayleigh-Chebyshev iteration, Sec. II B) on the columns
 * [col0, col0 + ncol) of row-major [N][ld] blocks:
 *     y = alpha (H x) + beta x + gamma prev + src_coef[col] src
 *  precision 0: x, prev, y complex128;  1: x, prev, src, y complex64
 *  prev_dev  NULL drops the gamma term;  src_dev NULL drops the source term
 *            (src needs precision 1 and src_coef_host, float64 [ld])
 *  y must not alias x, prev or src; columns outside the range are left
 *  unchanged.  Asynchronous on the handle's stream.  FP32 steps without a
 *  point mask, in the crystal or [110] frame and at B = 0 or in the
 *  symmetric gauge, with even ld and col0, run in the plane-marching kernel
 *  (TMA-staged z-planes); other steps in the per-point kernel.
 * Errors: INVALID_ARG (NULL or aliased blocks, ld outside 1..64, columns
 * outside the row, non-finite coefficients), STATE (fields not set). */
khp_status khp_filter_step(khp_handle h, const void* x_dev, const void* prev_dev, const void* src_dev,
                           const double* src_coef_host, void* y_dev, int ld, int col0, int ncol,
                           double alpha, double beta, double gamma, int precision);

/* The two dense contractions of the Rayleigh-Ritz step (Sec. II B), on the
 * handle's grid length N, for a block that is not the solver's own.
 *  khp_project: G = Y^H Y and (W_dev given) S = Y^H W, each m x m complex128
 *    row-major in host memory; both are formed from their upper triangles as
 *    Hermitian matrices (the solver's W is H Y).
 *  khp_rotate: X = Y Q and (W_dev given) HX = W Q, Q m x m complex128
 *    row-major in host memory; X may be Y and HX may be W (in place).
 *  Y_dev, W_dev, X_dev, HX_dev: complex128 [N][m] row-major on the device.
 *  method 0: tcgen05 tensor cores (accumulators in TMEM), exact split-digit
 *    BF16 products recombined in FP64 (m <= 32); 1: FP64 ALU; 2: the same
 *    split-digit products through mma.sync (m <= 32).  All synchronise the
 *    handle's stream; the first call allocates the handle's reduction
 *    scratch.
 * Errors: INVALID_ARG for NULL pointers, m outside 1..64, a bad method or
 * method 0 or 2 with m > 32; CUDA when a tensor-core pipeline wait of
 * method 0 ran out (bounded waits). */
khp_status khp_project(khp_handle h, const void* Y_dev, const void* W_dev, int m, int method,
                       double* G_host, double* S_host);
/* khp_project over `rows` rows instead of the handle's N (any block of
 * complex128 [rows][m], e.g. orbital-resolved or pair-density blocks of the
 * CI step); the handle supplies the stream and scratch. */
khp_status khp_project_rows(khp_handle h, const void* Y_dev, const void* W_dev, long long rows, int m,
                            int method, double* G_host, double* S_host);
khp_status khp_rotate(khp_handle h, const void* Y_dev, const void* W_dev, const double* Q_host,
                      int m, int method, void* X_dev, void* HX_dev);

/* Lowest opts->n_states eigenpairs (Sec. II B).
 *  evals_host  float64 [n_states], ascending
 *  evecs_dev   complex128 [N][n_states] row-major, orthonormal columns
 *  resid_host  optional float64 [n_states] residual norms ||H x - theta x||
 *  stats       optional
 * Returns NOT_CONVERGED (with the current Ritz pairs written) when max_iter
 * is reached before every residual is <= tol_ev.
 * The filter degree of an outer iteration is capped so that the filter
 * amplifies the bottom of the spectrum at most 1e4 times relative to the
 * filter interval (1e5 for precision 2), keeping the filtered block well
 * conditioned.  Environment: KHP_TRACE=1 prints one line per outer
 * iteration (2 adds every column's Ritz value and residual) to stderr;
 * KHP_AMP_CAP=<value > 1> replaces the amplification cap (tuning). */
khp_status khp_eigensolve(khp_handle h, const khp_solver_opts* opts, double* evals_host,
                          void* evecs_dev, double* resid_host, khp_stats* stats);

/* Flags of khp_eigensolve_batched. */
#define KHP_BATCH_GRAPH 1      /* capture every round of the batch into one CUDA graph */
#define KHP_BATCH_AUTOTUNE 2   /* choose block_m by timed trial solves (opts->block_m ignored) */
#define KHP_BATCH_GROUPED 4    /* one launch per filter step across the problems (precision 2) */

/* Poisson step of the Schroedinger-Poisson loop (Sec. II B).  On the
 * Schroedinger grid (nx, ny, nz, spacing h_nm), the potential phi [V] of the
 * hole density rho [nm^-3] is fixed at the gate points and has zero normal
 * flux at the box faces elsewhere:
 *     sum over in-box face neighbours n of (phi_p - phi_n) / h^2 = (e / eps) rho_p,
 *     eps = eps0 eps_r,  phi_p = phi_gate(p) at gates.
 * Every connected set of free points must touch a gate.  Solved by
 * preconditioned conjugate gradients on the device (the paper names no
 * solver): by default with a geometric multigrid V-cycle (cell-centred
 * 2x2x2 aggregation down to at most 64 cells, coarse cells that hold a gate
 * point are gates, the 7-point operator rediscretised at each spacing, two
 * weighted-Jacobi sweeps (0.8) before and after the coarse correction, a
 * dense solve on the coarsest level; FP32), else with the diagonal (Jacobi)
 * preconditioner; see khp_poisson_set_preconditioner. */
typedef struct khp_poisson_s* khp_poisson;

/* Preconditioners of the Poisson CG. */
#define KHP_POISSON_PRECOND_JACOBI 0
#define KHP_POISSON_PRECOND_MULTIGRID 1

/*  gate_mask_dev  uint8 [Np] device array, nonzero = gate point (copied)
 *  gate_phi_dev   float64 [Np] device array, gate potentials [V] (read at gates, copied)
 *  stream         cudaStream_t (as void*) for all work of this handle
 * Errors: INVALID_ARG for bad sizes, h or eps_r <= 0, NULL arrays. */
khp_status khp_poisson_create(khp_poisson* out, int nx, int ny, int nz, double h_nm, double eps_r,
                              const uint8_t* gate_mask_dev, const double* gate_phi_dev, void* stream);

/*  rho_dev   float64 [Np] hole density [nm^-3] (device)
 *  phi_dev   float64 [Np] (device): in = starting guess at the free points
 *            (e.g. zeros or the previous solution), out = phi [V]
 *  tol       stop when ||r|| <= tol ||b|| on the free points
 *  iterations, rel_residual  optional outputs
 * Synchronises the handle's stream.  Returns NOT_CONVERGED (phi holds the
 * last iterate) when max_iter is reached. */
khp_status khp_poisson_solve(khp_poisson p, const double* rho_dev, double* phi_dev, double tol, int max_iter,
                             int* iterations, double* rel_residual);

/* Solves of nrhs right-hand sides at once (the Coulomb potentials of the
 * CI's pair densities, the unit-occupation potentials of the relaxed SP
 * update): the CG runs them side by side in batches of up to 32, every
 * kernel launch covering the batch, until the largest relative residual of
 * the batch is at most tol.
 *  rho_dev   float64 [nrhs][Np] densities [nm^-3] (device)
 *  phi_dev   float64 [nrhs][Np] (device): in = starting guesses, out = phi [V]
 *  grounded  nonzero: gate potentials zero (the potential of the density
 *            alone); 0: the handle's gate potentials
 *  iterations      optional: the most CG iterations a batch took
 *  max_rel_residual optional: the largest relative residual
 * Synchronises the handle's stream.  Errors: INVALID_ARG (NULL arrays,
 * nrhs < 1, tol <= 0, max_iter < 1), OOM (the batch's vectors: about
 * 62 bytes per point and right-hand side, allocated on first use),
 * NOT_CONVERGED as khp_poisson_solve. */
khp_status khp_poisson_solve_many(khp_poisson p, const double* rho_dev, double* phi_dev, int nrhs, int grounded,
                                  double tol, int max_iter, int* iterations, double* max_rel_residual);

/* Selects the preconditioner of the handle's later solves
 * (KHP_POISSON_PRECOND_*; multigrid is the default).  The multigrid
 * hierarchy is built by khp_poisson_create: three FP32 vectors and a 16-bit
 * neighbour code per grid point, and about 1/7 of that again for the
 * coarse levels (the V-cycle runs in FP32; the CG's vectors and dot
 * products stay FP64).  Where it could not be built
 * (a grid that does not coarsen to 64 cells in 12 levels, or one without
 * gates) the solves use the Jacobi preconditioner.
 *  levels  optional output: the multigrid levels in use (0 = Jacobi)
 * Synchronises the handle's private stream when the choice changes.
 * Errors: INVALID_ARG (NULL handle, unknown kind). */
khp_status khp_poisson_set_preconditioner(khp_poisson p, int kind, int* levels);

/* Potential update of the loop: V = (1 - mix) V + mix (V_ext + phi), all
 * float64 [Np] device arrays (V_ext may be NULL), mix in (0, 1];
 * max_change (optional, host) = max |V_new - V_old|.  Synchronises. */
khp_status khp_sp_update(khp_poisson p, const double* V_ext_dev, const double* phi_dev, double mix, double* V_dev,
                         double* max_change);

/* Anderson-mixed potential update of the Schroedinger-Poisson loop (the
 * paper repeats the loop until convergence, Sec. II B, and names no scheme;
 * this type-II Anderson mixing is an addition).  With the residual
 * F_k = V_ext + phi - V_k of the fixed point and the differences
 * dV_i = V_{i+1} - V_i, dF_i = F_{i+1} - F_i of the last m = min(k, depth)
 * calls (kept on the handle):
 *     gamma   = argmin |F_k - dF gamma|_2   (m <= 8; tall-skinny QR of
 *               [dF | F] by Givens rotations on the device, the small
 *               factor's SVD on the host; minimum-norm solution with
 *               singular values <= eps max(Np, m) sigma_max dropped)
 *     V_{k+1} = V_k + beta F_k - sum_i gamma_i (dV_i + beta dF_i)
 * The first call after khp_poisson_create, khp_sp_anderson_reset or a
 * change of depth is the linear step V + beta F.  A zero history gives
 * gamma = 0, that step.
 *  V_ext_dev  float64 [Np] or NULL (zero);  phi_dev float64 [Np]
 *  V_dev      float64 [Np], updated in place
 *  max_change max |V_{k+1} - V_k| (host)
 * Synchronous.  Errors: INVALID_ARG (NULL, beta outside (0, 1], depth
 * outside 1..8), OOM (history buffers: (2 depth_max + 3) Np doubles). */
khp_status khp_sp_anderson(khp_poisson p, const double* V_ext_dev, const double* phi_dev, double beta, int depth,
                           double* V_dev, double* max_change);

/* Fermi level of the Schroedinger-Poisson loop (Sec. II B: the hole
 * density of the loop sums the states with Fermi-Dirac weights at the
 * device temperature; the number of holes is fixed).  Host-only, no device
 * work.
 *  E_host    float64 [n] level energies [eV] (any order)
 *  n_holes   number of holes, 0 < n_holes < n
 *  kT        thermal energy [eV], > 0
 *  mu_out    mu with sum_i 1 / (1 + exp((E_i - mu) / kT)) = n_holes
 *  occ_host  optional float64 [n] output, the occupations at mu
 * Safeguarded Newton iteration (bisection inside a bracket whenever the
 * Newton step leaves it or stalls); converges to rounding for any spread
 * of the levels.  Errors: INVALID_ARG (NULL, n < 1, kT <= 0, n_holes
 * outside (0, n), non-finite level). */
khp_status khp_fermi_level(const double* E_host, int n, double n_holes, double kT, double* mu_out,
                           double* occ_host);

/* Per-state densities of n states (the inputs of the relaxed-occupation
 * step below): dens_dev[i][p] = sum_b |psi_i(nb p + b)|^2, float64 [n][Np]
 * device (state-major), evecs_dev complex128 [N][n] row-major (N = nb Np;
 * nb = 6, or 3 for an H0 handle).  n in 1..64.  Asynchronous. */
khp_status khp_state_densities(khp_handle h, const void* evecs_dev, int n, double* dens_dev);

/* One Schroedinger-Poisson update with relaxed occupations.  The paper
 * repeats the loop until convergence (Sec. II B) at 1.5 K (Sec. III A);
 * there, fixed Fermi-Dirac occupations of the current levels let the holes
 * jump between near-degenerate wells from one iteration to the next.  Here
 * the occupations answer the new potential within the step, with the n
 * states of H(V) held fixed:
 *   Q_j   potential of a unit occupation of state j (density dens_j / h^3,
 *         gates grounded), phi_g the potential of the gates alone (CG on
 *         the device, the Q_j solved side by side as in
 *         khp_poisson_solve_many, each started from the previous call's);
 *   K_ij  = sum_p dens_i(p) Q_j(p),  e0_i = E_i + sum_p dens_i(p) (phi_g - (V - V_ext))(p);
 *   f     the Fermi-Dirac occupations of the levels eps = e0 + K f at the
 *         Fermi level holding n_holes (Newton's method on eps, host);
 *   phi   = phi_g + sum_j f_j Q_j.
 * The caller mixes V_ext + phi into V (khp_sp_update / khp_sp_anderson).
 * At a fixed point f are the Fermi-Dirac occupations of H(V).
 *  dens_dev   float64 [n][Np] from khp_state_densities (device)
 *  E_host     float64 [n] eigenvalues of the states [eV]
 *  V_dev, V_ext_dev  float64 [Np] the potential of the states and the
 *             external potential (NULL = 0) [eV]
 *  phi_dev    float64 [Np] output [V]
 *  tol        relative residual of the CG solves
 *  occ_host   optional float64 [n] output, the occupations; mu_out optional
 * Synchronous.  Errors: INVALID_ARG (NULL, n outside 1..64, kT <= 0,
 * n_holes outside (0, n), non-finite level), OOM (2 + n Np doubles on the
 * handle, and the batch vectors of khp_poisson_solve_many), NOT_CONVERGED
 * (a CG solve), BREAKDOWN (singular Newton system). */
khp_status khp_sp_relax_occupations(khp_poisson p, const double* dens_dev, const double* E_host, int n,
                                    double n_holes, double kT, const double* V_dev, const double* V_ext_dev,
                                    double* phi_dev, double tol, double* occ_host, double* mu_out);

/* Forget the Anderson history (start of a new self-consistent loop). */
khp_status khp_sp_anderson_reset(khp_poisson p);

khp_status khp_poisson_destroy(khp_poisson p);

/* Solve `count` independent problems (a gate-voltage / detuning sweep,
 * Sec. II C: the single-particle problem is re-solved for every detuning
 * point; grids may differ in size).  Every problem runs the same algorithm as
 * khp_eigensolve with the same options; the problems advance in lock-step
 * rounds (one outer iteration each, converged problems drop out), each
 * problem on its own internal stream so their kernels overlap.
 *  hs         count distinct handles on one device, fields set
 *  evals_host float64 [count][n_states]
 *  evecs_dev  count device pointers, each complex128 [N_i][n_states]
 *  resid_host optional float64 [count][n_states]
 *  stats      optional [count]
 *  flags      KHP_BATCH_GRAPH: every round is captured from a master stream
 *             (fork/join over the problems' streams) into one CUDA graph and
 *             launched once; the executable graph is updated in place when
 *             the round's topology is unchanged.
 *             KHP_BATCH_AUTOTUNE: block_m is chosen among n+4, n+8, n+12 by
 *             timed trial solves of the smallest problem.
 *             KHP_BATCH_GROUPED: in rounds where every active problem runs
 *             the defect-corrected FP32 filter (precision 2), the round runs
 *             on one stream and step k of all problems' filters is one
 *             launch of the plane-marching stencil whose work items are
 *             (problem, z-chunk, vector group, x-y tile), up to 8 problems
 *             per launch; the results equal the ungrouped ones bit for bit.
 *             Rounds it does not cover run as without the flag.
 * Warm starts are not accepted here.  Returns NOT_CONVERGED if any problem
 * hit max_iter (all results are still written). */
khp_status khp_eigensolve_batched(const khp_handle* hs, int count, const khp_solver_opts* opts,
                                  double* evals_host, void* const* evecs_dev, double* resid_host,
                                  khp_stats* stats, int flags);

/* Overlap (pair) densities of n states for the Coulomb integrals of the
 * configuration-interaction step (Sec. II C, Eqs. 13-15):
 *     rho_jl(p) = sum_b conj(psi_j(p, b)) psi_l(p, b)  for all ordered (j, l)
 * (per grid point, not divided by h^3).
 *  evecs_dev  complex128 [N][n] row-major (as returned by khp_eigensolve)
 *  rho_dev    complex128 [Np][n * n] row-major, pair index j n + l
 * Asynchronous on the handle's stream.  Errors: INVALID_ARG for NULL
 * pointers or n outside 1..64. */
khp_status khp_pair_densities(khp_handle h, const void* evecs_dev, int n, void* rho_dev);

/* First moments of m states about the box centre (the position operator
 * projected on them).  The eigenvectors of the projection along the dot
 * axis localise the bonding and anti-bonding doublets of a double dot on
 * the left and right dots, whose g-matrices give the g-tensors of Eq. 16
 * (Sec. III B):
 *     D[a][i][j] = sum_p r_a(p) sum_b conj(X_i(p, b)) X_j(p, b),
 *     r_a(p) = (i_a(p) - (n_a - 1) / 2) h   (nm),   a = x, y, z.
 *  X_dev   complex128 [N][m] row-major on the handle's device (N = bands Np)
 *  D_host  complex128 [3][m][m] (Hermitian), written before the call returns
 * Synchronous on the handle's stream.  Errors: INVALID_ARG for NULL
 * pointers or m outside 1..16. */
khp_status khp_position_moments(khp_handle h, const void* X_dev, int m, double* D_host);

/* Hole density (Sec. II B, fed to Poisson):
 *  rho_dev[p] = sum_i w_host[i] * sum_b |psi_i(6p+b)|^2   (discrete norm)
 *  evecs_dev complex128 [N][n] row-major.  Deterministic summation order. */
khp_status khp_density(khp_handle h, const void* evecs_dev, int n, const double* w_host,
                       double* rho_dev);

/* Hellmann-Feynman gradients of L(E_0..E_{n-1}) given dL/dE:
 *  dLdV_dev[p]         = sum_i g_i sum_b |psi_i(6p+b)|^2
 *  dLdstrain_dev[c][p] = sum_i g_i psi_i(p)^dag (dH'_PB/deps_c x 1) psi_i(p)
 *                        (NULL to skip)
 *  dLdalpha_host[g]    = sum_p dLdV[p] * levers_dev[g][p]  (n_gates >= 0)
 * evals_host are the eigenvalues belonging to evecs_dev; states closer than
 * 1e-6 eV form a cluster and g must be equal inside a cluster, else
 * KHP_ERR_DEGENERATE (the gradient of a split cluster is not defined). */
khp_status khp_eigs_backward(khp_handle h, const void* evecs_dev, const double* evals_host,
                             int n, const double* dLdE_host, double* dLdV_dev,
                             double* dLdstrain_dev, const double* levers_dev, int n_gates,
                             double* dLdalpha_host);

/* Allocation-free variant of khp_eigs_backward (the paper has no
 * counterpart; it exists for callers of this library).  Same arguments,
 * results and errors as khp_eigs_backward.  It is for callers that must not
 * see device memory allocated or freed during the call: a process whose
 * device memory is all owned by a pooling allocator, a latency-critical loop
 * where an allocation or free could synchronise the device, or a host that
 * forbids the library to hold device memory of its own between calls.
 * Instead of allocating its reduction scratch per call, it uses one fixed
 * array in device memory (KHP_NOALLOC_BLOCKS = 296 blocks x 16 gates of
 * partial sums plus 16 results, about 38 KB per GPU, held until the process
 * exits).  Limits: n_gates <= 16 (larger counts fail with
 * KHP_ERR_INVALID_ARG), n <= 64.
 *  - The first call on each device looks up the array's device address
 *    (cudaGetSymbolAddress) and caches it; make that first call before any
 *    stream capture.
 *  - All calls share the array: calls whose kernels overlap on the GPU
 *    (other streams or unordered host threads) race and must be serialised
 *    by the caller.
 *  - It runs on the handle's stream and synchronises it when n_gates > 0
 *    (it copies dL/dalpha to the host), so such calls cannot be captured
 *    into a CUDA graph; with n_gates = 0 a call can be captured once a
 *    first uncaptured call has been made on that device. */
khp_status khp_eigs_backward_noalloc(khp_handle h, const void* evecs_dev, const double* evals_host,
                                     int n, const double* dLdE_host, double* dLdV_dev,
                                     double* dLdstrain_dev, const double* levers_dev, int n_gates,
                                     double* dLdalpha_host);

/* Free the handle and its workspace (synchronises its stream). */
khp_status khp_destroy(khp_handle h);

/* Message of the last failure on the calling thread ("" if none). */
const char* khp_last_error(void);

/* Library version (major*10000 + minor*100 + patch). */
int khp_version(void);

#ifdef __cplusplus
}
#endif

#endif /* KHP_H */
