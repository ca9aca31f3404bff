// C ABI of the k.p hole eigensolver: handle life cycle, operator
// construction on the host (the constant 3x3 / 6x6 pieces of H_DKK, H_SOI,
// H'_PB and the Zeeman term), and the Chebyshev-filtered subspace iteration
// that drives the device kernels.
//
// Operator (paper Eqs. 2b, 5-6a; conventions where the paper is silent):
//   H = [C sum_ab D'_ijab k_a k_b + H'_PB,ij(eps(r)) + V(r) delta_ij] x 1_spin
//       + (Delta/3)(1 - L.sigma) + mu_B B.(gL L + 2 S)
// with C = hbar^2/2m0, D_iiii = g1+4g2, D_iijj = g1-2g2, D_ijij = D_ijji = 3g3,
// the Bir-Pikus tensor of the same form with l=-(a_v+2b), m=-(a_v-b),
// n=-sqrt3 d, both rotated into the grid frame on all four indices,
// (L_k)_ij = -i eps_kij, gL = 3 kappa - 1, k = -i grad discretised by central
// differences on 19 points, and Peierls phases exp(-i A(mid).(r'-r)/Phi0) on
// every link.
//
// Eigensolver (the Rayleigh-Chebyshev subspace iteration of Sec. II B):
//   X <- random (or warm start);  W = H X;  Rayleigh-Ritz
//   repeat:  Y = T_d((H - c)/e) X   (scaled three-term recurrence, fused stencil)
//            W = H Y
//            G = Y^H Y, S = Y^H W   (one pass)
//            S q = theta G q        (equilibrated Cholesky of G + Jacobi, one CTA)
//            X = Y Q, HX = W Q      (one pass, residual norms fused)
//   until ||HX_i - theta_i X_i|| <= tol for the wanted states.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "khp_common.cuh"
#include "khp_internal.h"

using namespace khp;
using cplx = std::complex<double>;

static thread_local std::string g_err;
static constexpr int kLzPartials = 296;

static khp_status fail(khp_status s, const std::string& msg) {
    g_err = msg;
    return s;
}

khp_status khp_set_error(khp_status s, const std::string& msg) { return fail(s, msg); }
void khp_clear_error() { g_err.clear(); }

#define CK(call)                                                                        \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess)                                                          \
            return fail(e_ == cudaErrorMemoryAllocation ? KHP_ERR_OOM : KHP_ERR_CUDA,   \
                        std::string(#call) + ": " + cudaGetErrorString(e_));            \
    } while (0)

#define CKS(expr)                        \
    do {                                 \
        khp_status s_ = (expr);          \
        if (s_ != KHP_OK) return s_;     \
    } while (0)

// ------------------------------------------------------ host operator set-up
namespace {

struct T4 {
    double v[3][3][3][3];
};

T4 luttinger(double g1, double g2, double g3) {
    T4 D{};
    for (int i = 0; i < 3; ++i) {
        D.v[i][i][i][i] = g1 + 4 * g2;
        for (int j = 0; j < 3; ++j)
            if (i != j) {
                D.v[i][i][j][j] = g1 - 2 * g2;
                D.v[i][j][i][j] = 3 * g3;
                D.v[i][j][j][i] = 3 * g3;
            }
    }
    return D;
}

T4 bir_pikus(double a_v, double b, double d) {
    const double l = -(a_v + 2 * b), m = -(a_v - b), n = -std::sqrt(3.0) * d;
    T4 D{};
    for (int i = 0; i < 3; ++i) {
        D.v[i][i][i][i] = l;
        for (int j = 0; j < 3; ++j)
            if (i != j) {
                D.v[i][i][j][j] = m;
                D.v[i][j][i][j] = n / 2;
                D.v[i][j][j][i] = n / 2;
            }
    }
    return D;
}

// D'_abcd = R_ai R_bj R_ck R_dl D_ijkl, done one index at a time
T4 rotate(const T4& D, const double* R) {
    T4 a{}, b{};
    for (int p = 0; p < 3; ++p) for (int j = 0; j < 3; ++j) for (int k = 0; k < 3; ++k) for (int l = 0; l < 3; ++l) {
        double s = 0; for (int i = 0; i < 3; ++i) s += R[p * 3 + i] * D.v[i][j][k][l]; a.v[p][j][k][l] = s; }
    for (int p = 0; p < 3; ++p) for (int q = 0; q < 3; ++q) for (int k = 0; k < 3; ++k) for (int l = 0; l < 3; ++l) {
        double s = 0; for (int j = 0; j < 3; ++j) s += R[q * 3 + j] * a.v[p][j][k][l]; b.v[p][q][k][l] = s; }
    for (int p = 0; p < 3; ++p) for (int q = 0; q < 3; ++q) for (int r = 0; r < 3; ++r) for (int l = 0; l < 3; ++l) {
        double s = 0; for (int k = 0; k < 3; ++k) s += R[r * 3 + k] * b.v[p][q][k][l]; a.v[p][q][r][l] = s; }
    for (int p = 0; p < 3; ++p) for (int q = 0; q < 3; ++q) for (int r = 0; r < 3; ++r) for (int t = 0; t < 3; ++t) {
        double s = 0; for (int l = 0; l < 3; ++l) s += R[t * 3 + l] * a.v[p][q][r][l]; b.v[p][q][r][t] = s; }
    return b;
}

// 3x3 (row-major) -> symmetric storage (00, 11, 22, 12, 02, 01)
void to_sym(const double M[3][3], double out[6]) {
    out[0] = M[0][0];
    out[1] = M[1][1];
    out[2] = M[2][2];
    out[3] = 0.5 * (M[1][2] + M[2][1]);
    out[4] = 0.5 * (M[0][2] + M[2][0]);
    out[5] = 0.5 * (M[0][1] + M[1][0]);
}

// Entries of the rotated operator pieces below 1e-14 of the largest entry
// are rounding residue of the rotation (exact zeros of the tensor form) and
// are set to zero, so that the stencil skips them.
void clean_small(double* v, int n) {
    double mx = 0.0;
    for (int i = 0; i < n; ++i) mx = std::max(mx, std::fabs(v[i]));
    for (int i = 0; i < n; ++i)
        if (std::fabs(v[i]) <= 1e-14 * mx) v[i] = 0.0;
}

void build_operator(khp_grid* g) {
    const khp_material& m = g->mat;
    const double C = KHP_HB2M, h2 = g->h * g->h;
    const T4 D = rotate(luttinger(m.gamma1, m.gamma2, m.gamma3), g->rot);
    double M[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double s = 0;
            for (int a = 0; a < 3; ++a) s += 2.0 * C * D.v[i][j][a][a] / h2;
            M[i][j] = s;
        }
    to_sym(M, g->center);
    // faces (pairs 0..2) and edges (pairs 3..8)
    for (int d = 0; d < 9; ++d) {
        const int off[3] = {pair_dx(d), pair_dy(d), pair_dz(d)};
        int ax[2], na = 0;
        for (int a = 0; a < 3; ++a)
            if (off[a] != 0) ax[na++] = a;
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                if (na == 1) {
                    M[i][j] = -C * D.v[i][j][ax[0]][ax[0]] / h2;
                } else {
                    const double sg = off[ax[0]] * off[ax[1]];
                    M[i][j] = -C * (D.v[i][j][ax[0]][ax[1]] + D.v[i][j][ax[1]][ax[0]]) * sg / (4.0 * h2);
                }
            }
        to_sym(M, g->hop[d]);
    }
    // strain derivative matrices per input component (xx,yy,zz,yz,xz,xy)
    const T4 E = rotate(bir_pikus(m.a_v, m.b, m.d), g->rot);
    const int pa[6] = {0, 1, 2, 1, 0, 0}, pb[6] = {0, 1, 2, 2, 2, 1};
    for (int c = 0; c < 6; ++c) {
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
                M[i][j] = pa[c] == pb[c] ? E.v[i][j][pa[c]][pa[c]]
                                         : E.v[i][j][pa[c]][pb[c]] + E.v[i][j][pb[c]][pa[c]];
        to_sym(M, g->De[c]);
    }
    clean_small(&g->hop[0][0], 9 * 6);
    clean_small(g->center, 6);
    clean_small(&g->De[0][0], 6 * 6);
    // spin-orbit + Zeeman on index 3 s + o
    cplx L[3][3][3] = {};
    const double eps[3][3][3] = {{{0, 0, 0}, {0, 0, 1}, {0, -1, 0}},
                                 {{0, 0, -1}, {0, 0, 0}, {1, 0, 0}},
                                 {{0, 1, 0}, {-1, 0, 0}, {0, 0, 0}}};
    for (int k = 0; k < 3; ++k)
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) L[k][i][j] = cplx(0.0, -eps[k][i][j]);
    const cplx sig[3][2][2] = {{{0, 1}, {1, 0}},
                               {{0, cplx(0, -1)}, {cplx(0, 1), 0}},
                               {{1, 0}, {0, -1}}};
    const double gL = 3.0 * m.kappa - 1.0;
    for (int b1 = 0; b1 < 6; ++b1)
        for (int b2 = 0; b2 < 6; ++b2) {
            const int s1 = b1 / 3, o1 = b1 % 3, s2 = b2 / 3, o2 = b2 % 3;
            cplx v = (b1 == b2) ? cplx(m.delta_so / 3.0, 0) : cplx(0, 0);
            for (int k = 0; k < 3; ++k) {
                v -= (m.delta_so / 3.0) * sig[k][s1][s2] * L[k][o1][o2];
                cplx z = 0;
                if (s1 == s2) z += gL * L[k][o1][o2];
                if (o1 == o2) z += sig[k][s1][s2];
                v += KHP_MU_B * g->B[k] * z;
            }
            // the spin-independent H0 has neither spin-orbit nor Zeeman term
            g->soz_re[b1][b2] = g->nb == 3 ? 0.0 : v.real();
            g->soz_im[b1][b2] = g->nb == 3 ? 0.0 : v.imag();
        }
}

double sym_rowsum_max(const double s[6]) {
    const double r0 = std::fabs(s[0]) + std::fabs(s[5]) + std::fabs(s[4]);
    const double r1 = std::fabs(s[5]) + std::fabs(s[1]) + std::fabs(s[3]);
    const double r2 = std::fabs(s[4]) + std::fabs(s[3]) + std::fabs(s[2]);
    return std::max(r0, std::max(r1, r2));
}

// Stencil coefficients scaled by alpha (the kernel computes
// alpha*H x + beta*x + gamma*prev with alpha folded in).
template <typename R>
void fill_coeffs(const khp_grid* g, Coeffs<R>& c, double alpha) {
    for (int d = 0; d < 9; ++d) {
        c.hop_nz[d] = 0;
        for (int k = 0; k < 6; ++k) {
            c.hop[d][k] = (R)(alpha * g->hop[d][k]);
            if (g->hop[d][k] != 0.0) c.hop_nz[d] |= 1u << k;
        }
    }
    for (int i = 0; i < 6; ++i) {
        c.soz_nz[i] = 0;
        for (int j = 0; j < 6; ++j) {
            c.soz_re[i][j] = (R)(alpha * g->soz_re[i][j]);
            c.soz_im[i][j] = (R)(alpha * g->soz_im[i][j]);
            if (g->soz_re[i][j] != 0.0) c.soz_nz[i] |= 1u << (2 * j);
            if (g->soz_im[i][j] != 0.0) c.soz_nz[i] |= 2u << (2 * j);
        }
    }
    // on-site orbital block: centre pattern, V on the diagonal, strain
    c.onsite_nz = 0;
    for (int k = 0; k < 6; ++k) {
        bool nz = k < 3 || g->center[k] != 0.0;
        if (g->has_strain)
            for (int cc = 0; cc < 6; ++cc) nz = nz || g->De[cc][k] != 0.0;
        if (nz) c.onsite_nz |= 1u << k;
    }
    c.pair_phase = g->pair_phase;
}

// Pairs whose Peierls phase vanishes identically on the whole grid: in the
// symmetric gauge phi_d = (r - c).(delta_d x B) / (2 Phi0) vanishes iff
// delta_d x B = 0; in the Landau gauge A.delta = dy (Bz x - Bx z) - dz By x.
unsigned phase_pairs(const double B[3], int gauge) {
    unsigned m = 0;
    for (int d = 0; d < 9; ++d) {
        const double dx = pair_dx(d), dy = pair_dy(d), dz = pair_dz(d);
        bool nz;
        if (gauge == 0) {
            const double cx = dy * B[2] - dz * B[1], cy = dz * B[0] - dx * B[2], cz = dx * B[1] - dy * B[0];
            nz = cx != 0.0 || cy != 0.0 || cz != 0.0;
        } else {
            nz = (dy != 0.0 && (B[2] != 0.0 || B[0] != 0.0)) || (dz != 0.0 && B[1] != 0.0);
        }
        if (nz) m |= 1u << d;
    }
    return m;
}

template <typename R>
khp_status apply_op(khp_grid* g, const cx_t<R>* x, const cx_t<R>* prev, cx_t<R>* y, int ld,
                    int col0, int ncol, double alpha, double beta, double gamma) {
    StencilArgs<R> a;
    a.nx = g->nx; a.ny = g->ny; a.nz = g->nz;
    a.ld = ld; a.col0 = col0; a.ncol = ncol;
    a.alpha = (R)alpha; a.beta = (R)beta; a.gamma = (R)gamma;
    a.x = x; a.prev = prev; a.y = y;
    if constexpr (sizeof(R) == 8) {
        a.onsite = (const R*)g->onsite64;
        a.phase = (const cx_t<R>*)(g->has_phase ? g->phase64 : nullptr);
    } else {
        a.onsite = (const R*)g->onsite32;
        a.phase = (const cx_t<R>*)(g->has_phase ? g->phase32 : nullptr);
    }
    a.mask = g->mask;
    a.phase_mode = g->has_phase ? g->phase_mode : PH_NONE;
    a.src = nullptr;
    a.nb = g->nb;
    a.err = g->dflag;
    fill_coeffs<R>(g, a.c, alpha);
    CK(launch_stencil<R>(a, g->stream));
    g->launches += 1;
    return KHP_OK;
}

void free_ws(khp_grid* g) {
    for (int i = 0; i < 4; ++i) { if (g->blk64[i]) cudaFree(g->blk64[i]); g->blk64[i] = nullptr; }
    for (int i = 0; i < 4; ++i) { if (g->blk32[i]) cudaFree(g->blk32[i]); g->blk32[i] = nullptr; }
    if (g->partial) cudaFree(g->partial);
    g->partial = nullptr;
    g->ws_m = 0;
    g->ws_has32 = 0;
}

khp_status ensure_ws(khp_grid* g, int m, bool need32) {
    if (g->ws_m >= m && (!need32 || g->ws_has32)) return KHP_OK;
    const int mm = std::max(m, g->ws_m);
    const bool w32 = need32 || g->ws_has32;
    CK(cudaStreamSynchronize(g->stream));
    free_ws(g);
    for (int i = 0; i < 4; ++i) CK(cudaMalloc(&g->blk64[i], sizeof(double2) * g->n * mm));
    if (w32)
        for (int i = 0; i < 4; ++i) CK(cudaMalloc(&g->blk32[i], sizeof(float2) * g->n * mm));
    const int nblk = dense_blocks(g->n);
    g->partial_elems = std::max(gram_partial_elems(KHP_MAX_M, nblk), (size_t)nblk * KHP_MAX_GATES);
    CK(cudaMalloc(&g->partial, sizeof(double2) * g->partial_elems));
    g->ws_m = mm;
    g->ws_has32 = w32;
    return KHP_OK;
}

// the reduction scratch alone (the projection entry points need no blocks)
khp_status ensure_partial(khp_grid* g) {
    if (g->partial) return KHP_OK;
    const int nblk = dense_blocks(g->n);
    g->partial_elems = std::max(gram_partial_elems(KHP_MAX_M, nblk), (size_t)nblk * KHP_MAX_GATES);
    CK(cudaMalloc(&g->partial, sizeof(double2) * g->partial_elems));
    return KHP_OK;
}

bool finite_all(const double* v, int n) {
    for (int i = 0; i < n; ++i)
        if (!std::isfinite(v[i])) return false;
    return true;
}

// Algorithmic work of one filter step at one interior point for one vector:
// the sparse product H x counted as 8 flop per complex and 4 per real
// nonzero of the point's 6 rows, plus 10 flop per component for the
// three-term update; bytes: Y_k, Y_k-1 read and Y_k+1 written once, and the
// per-point field tables (on-site 3x3, link phases) shared by the m vectors.
void op_counts(const khp_grid* g, int m, double* flops, double* b64, double* b32) {
    double f = 0.0;
    const int nb = g->nb;
    for (int b1 = 0; b1 < nb; ++b1)
        for (int b2 = 0; b2 < nb; ++b2) {
            const int s1 = b1 / 3, o1 = b1 % 3, s2 = b2 / 3, o2 = b2 % 3;
            const bool cplx_nz = g->soz_im[b1][b2] != 0.0;
            bool nz = g->soz_re[b1][b2] != 0.0 || cplx_nz;
            if (s1 == s2) {
                // centre + V (diagonal) + strain on the orbital block
                static const int sidx[3][3] = {{0, 5, 4}, {5, 1, 3}, {4, 3, 2}};
                const int k = sidx[o1][o2];
                bool onz = o1 == o2 || g->center[k] != 0.0;
                if (g->has_strain)
                    for (int c = 0; c < 6; ++c) onz = onz || g->De[c][k] != 0.0;
                nz = nz || onz;
            }
            if (nz) f += cplx_nz ? 8.0 : 4.0;
        }
    for (int d = 0; d < 9; ++d) {
        const double* h = g->hop[d];
        int nz = 0;
        for (int k = 0; k < 3; ++k) nz += h[k] != 0.0;
        for (int k = 3; k < 6; ++k) nz += 2 * (h[k] != 0.0);
        // two links (+/-), nb / 3 spins; complex entries when B != 0
        f += 2.0 * (nb / 3) * nz * (g->has_phase ? 8.0 : 4.0);
    }
    f += nb * 10.0;
    *flops = f;
    const double fields64 = 6 * 8.0 + (g->has_phase ? 18 * 16.0 : 0.0);
    *b64 = 3 * 16.0 * nb + fields64 / m;
    *b32 = 3 * 8.0 * nb + 0.5 * fields64 / m;
}

// Upper bound of the spectrum for the filter interval: k-step Lanczos from a
// random vector, bound = largest Ritz value + |beta_k|, never above the
// Gershgorin bound.  Uses the first N entries of the four workspace blocks.
khp_status lanczos_issue(khp_grid* g, int k, unsigned long long seed) {
    double* partial = g->lz;
    double* alpha = g->lz + kLzPartials;
    double* beta = alpha + KHP_MAX_M;
    double2* Wv = g->blk64[0];
    double2* P = g->blk64[1];
    double2* Cc = g->blk64[2];
    double2* Nn = g->blk64[3];
    const long long n = g->n;
    CK(launch_random_fill(Cc, n, 1, 0, 1, seed ^ 0x5bd1e995ULL, g->mask, g->stream, g->nb));
    CK(lanczos_norm(Cc, n, partial, beta, g->stream));
    CK(lanczos_scale(Cc, Cc, beta, n, g->stream));
    g->launches += 4;
    for (int j = 0; j < k; ++j) {
        CKS(apply_op<double>(g, Cc, nullptr, Wv, 1, 0, 1, 1.0, 0.0, 0.0));
        CK(lanczos_dot(Cc, Wv, n, partial, alpha + j, g->stream));
        CK(lanczos_orth(Wv, Cc, j > 0 ? P : nullptr, alpha + j, beta + j, beta + j + 1, n, partial, g->stream));
        CK(lanczos_scale(Nn, Wv, beta + j + 1, n, g->stream));
        g->launches += 5;
        double2* t = P; P = Cc; Cc = Nn; Nn = t;
    }
    double2* G = g->small;
    double2* S = g->small + k * k;
    double2* Q = g->small + 2 * k * k;
    double* th = g->dvec;
    CK(lanczos_tridiag(alpha, beta + 1, k, G, S, g->stream));
    CK(cudaMemsetAsync(g->dflag, 0, sizeof(int), g->stream));
    CK(launch_small(G, S, k, 1, Q, th, g->dflag, g->stream));
    g->launches += 2;
    double* hp = g->host_pinned;
    CK(cudaMemcpyAsync(hp, th + k - 1, sizeof(double), cudaMemcpyDeviceToHost, g->stream));
    CK(cudaMemcpyAsync(hp + 1, beta + k, sizeof(double), cudaMemcpyDeviceToHost, g->stream));
    CK(cudaMemcpyAsync(hp + 2, th, sizeof(double), cudaMemcpyDeviceToHost, g->stream));
    return KHP_OK;
}

// after the stream is synchronised: bounds from the pinned copies
void lanczos_finish(khp_grid* g, double* out, double* out_lo) {
    const double* hp = g->host_pinned;
    const double b = hp[0] + std::fabs(hp[1]);
    *out = std::isfinite(b) ? std::min(b, g->onsite_absmax) : g->onsite_absmax;
    // lower estimate of the spectrum (smallest Ritz value), used to cap the
    // filter amplification and as the scaling point
    const double lo = hp[2];
    *out_lo = std::isfinite(lo) ? std::max(lo, -g->onsite_absmax) : -g->onsite_absmax;
}

}  // namespace

// ====================================================================== ABI
extern "C" {

int khp_version(void) { return 100; }

const char* khp_last_error(void) { return g_err.c_str(); }

static khp_status create_grid(khp_handle* out, int nx, int ny, int nz, double h_nm,
                              const khp_material* mat, const double rot[9], const uint8_t* mask_dev,
                              void* stream, int nb) {
    g_err.clear();
    if (!out) return fail(KHP_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (nx < 1 || ny < 1 || nz < 1) return fail(KHP_ERR_INVALID_ARG, "grid sizes must be >= 1");
    if (!(h_nm > 0.0) || !std::isfinite(h_nm)) return fail(KHP_ERR_INVALID_ARG, "h must be > 0");
    if (!mat) return fail(KHP_ERR_INVALID_ARG, "material is NULL");
    if (!finite_all(&mat->gamma1, 8)) return fail(KHP_ERR_INVALID_ARG, "material has non-finite entries");
    const long long np = (long long)nx * ny * nz;
    if (np > (1LL << 31) / 6) return fail(KHP_ERR_INVALID_ARG, "grid too large");
    double R[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
    if (rot) {
        for (int i = 0; i < 9; ++i) R[i] = rot[i];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                double s = 0;
                for (int k = 0; k < 3; ++k) s += R[a * 3 + k] * R[b * 3 + k];
                if (std::fabs(s - (a == b ? 1.0 : 0.0)) > 1e-10)
                    return fail(KHP_ERR_INVALID_ARG, "rot is not orthonormal");
            }
    }
    khp_grid* g = new khp_grid();
    std::memset(g, 0, sizeof(khp_grid));
    g->nx = nx; g->ny = ny; g->nz = nz; g->np = np; g->nb = nb; g->n = (long long)nb * np; g->h = h_nm;
    g->mat = *mat;
    std::memcpy(g->rot, R, sizeof(R));
    g->stream = (cudaStream_t)stream;
    cudaGetDevice(&g->device);
    build_operator(g);
    auto bail = [&](khp_status s) { khp_destroy(g); return s; };
    cudaError_t e;
    if ((e = cudaMalloc(&g->onsite64, sizeof(double) * 6 * np)) != cudaSuccess ||
        (e = cudaMalloc(&g->onsite32, sizeof(float) * 6 * np)) != cudaSuccess ||
        (e = cudaMalloc(&g->dvec, sizeof(double) * 8 * KHP_MAX_M)) != cudaSuccess ||
        (e = cudaMalloc(&g->dflag, sizeof(int) * 8)) != cudaSuccess ||
        (e = cudaMalloc(&g->small, sizeof(double2) * 4 * KHP_MAX_M * KHP_MAX_M)) != cudaSuccess ||
        (e = cudaMalloc(&g->lz, sizeof(double) * (kLzPartials + 4 * KHP_MAX_M))) != cudaSuccess ||
        (e = cudaMallocHost(&g->host_pinned, sizeof(double) * 8 * KHP_MAX_M)) != cudaSuccess)
        return bail(fail(e == cudaErrorMemoryAllocation ? KHP_ERR_OOM : KHP_ERR_CUDA,
                         std::string("allocation: ") + cudaGetErrorString(e)));
    for (int k = 0; k < 5 && e == cudaSuccess; ++k) e = cudaEventCreate(&g->evp[k]);
    if (e != cudaSuccess || (e = cudaEventCreate(&g->ev0)) != cudaSuccess || (e = cudaEventCreate(&g->ev1)) != cudaSuccess)
        return bail(fail(KHP_ERR_CUDA, std::string("event: ") + cudaGetErrorString(e)));
    if ((e = prepare_oz()) != cudaSuccess || (e = prepare_tc()) != cudaSuccess)
        return bail(fail(KHP_ERR_CUDA, std::string("projection set-up: ") + cudaGetErrorString(e)));
    if ((e = prepare_plane()) != cudaSuccess)
        return bail(fail(KHP_ERR_CUDA, std::string("stencil set-up: ") + cudaGetErrorString(e)));
    if (mask_dev) {
        if ((e = cudaMalloc(&g->mask, np)) != cudaSuccess ||
            (e = cudaMemcpyAsync(g->mask, mask_dev, np, cudaMemcpyDeviceToDevice, g->stream)) != cudaSuccess)
            return bail(fail(KHP_ERR_CUDA, std::string("mask copy: ") + cudaGetErrorString(e)));
    }
    *out = g;
    return KHP_OK;
}

khp_status khp_create_grid(khp_handle* out, int nx, int ny, int nz, double h_nm,
                           const khp_material* mat, const double rot[9], const uint8_t* mask_dev,
                           void* stream) {
    return create_grid(out, nx, ny, nz, h_nm, mat, rot, mask_dev, stream, 6);
}

khp_status khp_create_grid_h0(khp_handle* out, int nx, int ny, int nz, double h_nm,
                              const khp_material* mat, const double rot[9], const uint8_t* mask_dev,
                              void* stream) {
    return create_grid(out, nx, ny, nz, h_nm, mat, rot, mask_dev, stream, 3);
}

khp_status khp_destroy(khp_handle g) {
    if (!g) return KHP_OK;
    cudaStreamSynchronize(g->stream);
    if (g->coarse) {
        // the coarse handle may still name a stream of an earlier call: it
        // works on the fine handle's stream
        g->coarse->stream = g->stream;
        khp_destroy(g->coarse);
    }
    if (g->coarse_x) cudaFree(g->coarse_x);
    free_ws(g);
    if (g->onsite64) cudaFree(g->onsite64);
    if (g->onsite32) cudaFree(g->onsite32);
    if (g->phase64) cudaFree(g->phase64);
    if (g->phase32) cudaFree(g->phase32);
    if (g->mask) cudaFree(g->mask);
    if (g->dvec) cudaFree(g->dvec);
    if (g->dflag) cudaFree(g->dflag);
    if (g->small) cudaFree(g->small);
    if (g->lz) cudaFree(g->lz);
    if (g->host_pinned) cudaFreeHost(g->host_pinned);
    if (g->ev0) cudaEventDestroy(g->ev0);
    if (g->ev1) cudaEventDestroy(g->ev1);
    for (int k = 0; k < 5; ++k)
        if (g->evp[k]) cudaEventDestroy(g->evp[k]);
    delete g;
    return KHP_OK;
}

// Gershgorin upper bound of the spectrum once the on-site block is set (and
// the device flag word of the field set-up, when bad is given)
static khp_status finish_fields(khp_grid* g, int* bad) {
    double* partial = g->dvec + 2 * KHP_MAX_M;   // 6*KHP_MAX_M doubles available
    const int nb = 4 * KHP_MAX_M;
    CK(launch_onsite_rowmax(g, partial, nb, g->dvec));
    CK(cudaMemcpyAsync(g->host_pinned, g->dvec, sizeof(double), cudaMemcpyDeviceToHost, g->stream));
    if (bad) CK(cudaMemcpyAsync(bad, g->dflag, sizeof(int), cudaMemcpyDeviceToHost, g->stream));
    CK(cudaStreamSynchronize(g->stream));
    if (bad && *bad) return KHP_OK;
    double soz = 0;
    for (int b = 0; b < 6; ++b) {
        double s = 0;
        for (int b2 = 0; b2 < 6; ++b2) s += std::hypot(g->soz_re[b][b2], g->soz_im[b][b2]);
        soz = std::max(soz, s);
    }
    double hops = 0;
    for (int d = 0; d < 9; ++d) hops += 2.0 * sym_rowsum_max(g->hop[d]);
    g->onsite_absmax = g->host_pinned[0] + soz + hops;
    g->fields_set = true;
    g->bound_valid = false;
    return KHP_OK;
}

// The coarse grid of the coarse-grid start: every second point at twice the
// spacing, the same material, frame, field and gauge (symmetric gauge about
// the fine grid's centre), on-site block restricted from the fine one.
static khp_status coarse_prepare(khp_grid* g) {
    if (!g->coarse) {
        khp_handle gc = nullptr;
        CKS(create_grid(&gc, g->nx / 2, g->ny / 2, g->nz / 2, 2.0 * g->h, &g->mat, g->rot, nullptr, g->stream,
                        g->nb));
        g->coarse = gc;
        if (g->mask) CK(cudaMalloc(&gc->mask, gc->np));
        gc->ctr[0] = 0.5 * (g->nx + 1) * g->h;
        gc->ctr[1] = 0.5 * (g->ny + 1) * g->h;
        gc->ctr[2] = 0.5 * (g->nz + 1) * g->h;
        gc->ctr_set = 1;
    }
    if (g->coarse_valid) return KHP_OK;
    khp_grid* gc = g->coarse;
    for (int k = 0; k < 3; ++k) gc->B[k] = g->B[k];
    gc->gauge = g->gauge;
    gc->has_phase = g->has_phase;
    gc->phase_mode = g->phase_mode;
    gc->pair_phase = g->pair_phase;
    gc->has_strain = g->has_strain;
    build_operator(gc);
    if (gc->has_phase && !gc->phase64) {
        CK(cudaMalloc(&gc->phase64, sizeof(double2) * 18 * gc->np));
        CK(cudaMalloc(&gc->phase32, sizeof(float2) * 18 * gc->np));
    }
    CK(launch_restrict_onsite(g, gc));
    CK(launch_phase_setup(gc));
    CKS(finish_fields(gc, nullptr));
    g->coarse_valid = true;
    return KHP_OK;
}

// Whether a block of m columns can start from the coarse grid: the coarse
// block (m + extra columns) fits the library's width and the coarse grid has
// at least 4 (m + extra) unknowns.
static bool coarse_eligible(const khp_grid* g, int m, int extra) {
    const long long npc = (long long)(g->nx / 2) * (g->ny / 2) * (g->nz / 2);
    return m + extra <= KHP_MAX_M && npc >= 1 && (long long)g->nb * npc >= 4LL * (m + extra);
}

// Options of the coarse solve for a fine solve with options o and width m:
// degree 120 (plain) or 60 (defect-corrected FP32), tolerance max(tol, 1e-3
// eV), block m + 8 (measured at C2: a tighter coarse tolerance does not
// improve the fine start, whose residuals are set by the difference of the
// two discretisations); KHP_COARSE="degree,tol_ev,extra_columns" in the
// environment replaces them (tuning).
static khp_solver_opts coarse_opts(const khp_solver_opts& o, int m) {
    int cdeg = o.precision == 0 ? 120 : 60, cextra = 8;
    double ctol = 1e-3;
    if (const char* cs = std::getenv("KHP_COARSE")) {
        int d = 0, x = 0;
        double t = 0.0;
        if (std::sscanf(cs, "%d,%lf,%d", &d, &t, &x) == 3 && d >= 1 && t > 0.0 && x >= 2 && (x % 2) == 0) {
            cdeg = d;
            ctol = t;
            cextra = x;
        }
    }
    khp_solver_opts oc{};
    oc.n_states = m;
    oc.block_m = m + cextra;
    oc.degree = cdeg;
    oc.max_iter = 60;
    oc.precision = o.precision == 0 ? 0 : 2;
    oc.refine_sweeps = o.refine_sweeps;
    oc.tol_ev = std::max(o.tol_ev, ctol);
    oc.seed = o.seed;
    oc.projections = o.projections;
    return oc;
}

static khp_status coarse_block(khp_grid* g, int m) {
    if (g->coarse_m >= m) return KHP_OK;
    if (g->coarse_x) cudaFree(g->coarse_x);
    g->coarse_x = nullptr;
    g->coarse_m = 0;
    CK(cudaMalloc(&g->coarse_x, sizeof(double2) * g->coarse->n * m));
    g->coarse_m = m;
    return KHP_OK;
}

khp_status khp_set_potential_strain_field(khp_handle g, const double* V_dev, const double* strain_dev,
                                          const double* levers_dev, const double* alpha_host,
                                          int n_gates, const double* B_host, int gauge) {
    g_err.clear();
    if (!g) return fail(KHP_ERR_INVALID_ARG, "handle is NULL");
    if (!V_dev) return fail(KHP_ERR_INVALID_ARG, "V is NULL");
    if (gauge != 0 && gauge != 1) return fail(KHP_ERR_INVALID_ARG, "gauge must be 0 or 1");
    if (n_gates < 0 || n_gates > KHP_MAX_GATES) return fail(KHP_ERR_INVALID_ARG, "n_gates out of range");
    if (n_gates > 0 && (!levers_dev || !alpha_host))
        return fail(KHP_ERR_INVALID_ARG, "levers and alpha required when n_gates > 0");
    if (n_gates > 0 && !finite_all(alpha_host, n_gates)) return fail(KHP_ERR_INVALID_ARG, "alpha non-finite");
    double B[3] = {0, 0, 0};
    if (B_host) {
        if (!finite_all(B_host, 3)) return fail(KHP_ERR_INVALID_ARG, "B non-finite");
        for (int k = 0; k < 3; ++k) B[k] = B_host[k];
        if (g->nb == 3 && (B[0] != 0.0 || B[1] != 0.0 || B[2] != 0.0))
            return fail(KHP_ERR_INVALID_ARG, "the spin-independent H0 has no magnetic field: B must be zero");
    }
    for (int k = 0; k < 3; ++k) g->B[k] = B[k];
    g->gauge = gauge;
    g->has_phase = (B[0] != 0.0 || B[1] != 0.0 || B[2] != 0.0);
    g->phase_mode = !g->has_phase ? PH_NONE : (gauge == 0 ? PH_SYM : PH_GEN);
    g->pair_phase = g->has_phase ? phase_pairs(B, gauge) : 0u;
    build_operator(g);
    if (g->has_phase && !g->phase64) {
        CK(cudaMalloc(&g->phase64, sizeof(double2) * 18 * g->np));
        CK(cudaMalloc(&g->phase32, sizeof(float2) * 18 * g->np));
    }
    CK(cudaMemsetAsync(g->dflag, 0, sizeof(int) * 8, g->stream));
    g->has_strain = strain_dev != nullptr;
    CK(launch_field_setup(g, V_dev, strain_dev, n_gates ? levers_dev : nullptr, alpha_host, n_gates, g->dflag));
    g->coarse_valid = false;
    int bad = 0;
    CKS(finish_fields(g, &bad));
    if (bad) {
        g->fields_set = false;
        return fail(KHP_ERR_INVALID_ARG, "non-finite value in V, strain or levers");
    }
    return KHP_OK;
}

khp_status khp_apply(khp_handle g, const void* X_dev, void* Y_dev, int m, int precision) {
    g_err.clear();
    if (!g) return fail(KHP_ERR_INVALID_ARG, "handle is NULL");
    if (!g->fields_set) return fail(KHP_ERR_STATE, "fields not set");
    if (!X_dev || !Y_dev) return fail(KHP_ERR_INVALID_ARG, "X or Y is NULL");
    if (m < 1 || m > KHP_MAX_M) return fail(KHP_ERR_INVALID_ARG, "m out of range 1..64");
    if (precision == 0)
        return apply_op<double>(g, (const double2*)X_dev, nullptr, (double2*)Y_dev, m, 0, m, 1.0, 0.0, 0.0);
    if (precision == 1)
        return apply_op<float>(g, (const float2*)X_dev, nullptr, (float2*)Y_dev, m, 0, m, 1.0, 0.0, 0.0);
    return fail(KHP_ERR_INVALID_ARG, "precision must be 0 or 1");
}

khp_status khp_filter_step(khp_handle g, const void* x_dev, const void* prev_dev, const void* src_dev,
                           const double* src_coef_host, void* y_dev, int ld, int col0, int ncol, double alpha,
                           double beta, double gamma, int precision) {
    g_err.clear();
    if (!g) return fail(KHP_ERR_INVALID_ARG, "handle is NULL");
    if (!g->fields_set) return fail(KHP_ERR_STATE, "fields not set");
    if (!x_dev || !y_dev) return fail(KHP_ERR_INVALID_ARG, "x or y is NULL");
    if (x_dev == y_dev || (prev_dev && prev_dev == y_dev) || (src_dev && src_dev == y_dev))
        return fail(KHP_ERR_INVALID_ARG, "y must not alias x, prev or src");
    if (ld < 1 || ld > KHP_MAX_M) return fail(KHP_ERR_INVALID_ARG, "ld out of range 1..64");
    if (col0 < 0 || ncol < 1 || col0 + ncol > ld) return fail(KHP_ERR_INVALID_ARG, "columns outside the row");
    if (precision != 0 && precision != 1) return fail(KHP_ERR_INVALID_ARG, "precision must be 0 or 1");
    if (src_dev && (precision != 1 || !src_coef_host))
        return fail(KHP_ERR_INVALID_ARG, "src needs precision 1 and src_coef");
    const double sc[3] = {alpha, beta, gamma};
    if (!finite_all(sc, 3) || (src_dev && !finite_all(src_coef_host, ld)))
        return fail(KHP_ERR_INVALID_ARG, "non-finite coefficient");
    if (precision == 0) {
        StencilArgs<double> a;
        a.nx = g->nx; a.ny = g->ny; a.nz = g->nz;
        a.ld = ld; a.col0 = col0; a.ncol = ncol;
        a.alpha = alpha; a.beta = beta; a.gamma = gamma;
        a.x = (const double2*)x_dev; a.prev = (const double2*)prev_dev; a.y = (double2*)y_dev;
        a.onsite = g->onsite64;
        a.phase = g->has_phase ? g->phase64 : nullptr;
        a.phase_mode = g->has_phase ? g->phase_mode : PH_NONE;
        a.mask = g->mask; a.src = nullptr; a.nb = g->nb; a.err = g->dflag;
        fill_coeffs<double>(g, a.c, alpha);
        CK(launch_stencil<double>(a, g->stream));
    } else {
        StencilArgs<float> a;
        a.nx = g->nx; a.ny = g->ny; a.nz = g->nz;
        a.ld = ld; a.col0 = col0; a.ncol = ncol;
        a.alpha = (float)alpha; a.beta = (float)beta; a.gamma = (float)gamma;
        a.x = (const float2*)x_dev; a.prev = (const float2*)prev_dev; a.y = (float2*)y_dev;
        a.onsite = g->onsite32;
        a.phase = (const float2*)(g->has_phase ? g->phase32 : nullptr);
        a.phase_mode = g->has_phase ? g->phase_mode : PH_NONE;
        a.mask = g->mask; a.src = (const float2*)src_dev; a.nb = g->nb; a.err = g->dflag;
        for (int c = 0; c < 64; ++c) a.src_coef[c] = (src_dev && c < ld) ? (float)src_coef_host[c] : 0.f;
        fill_coeffs<float>(g, a.c, alpha);
        CK(launch_stencil<float>(a, g->stream));
    }
    g->launches += 1;
    return KHP_OK;
}

khp_status khp_project_rows(khp_handle g, const void* Y_dev, const void* W_dev, long long rows, int m, int method,
                            double* G_host, double* S_host) {
    g_err.clear();
    if (!g) return fail(KHP_ERR_INVALID_ARG, "handle is NULL");
    if (rows < 1) return fail(KHP_ERR_INVALID_ARG, "rows must be >= 1");
    if (!Y_dev || !G_host || (W_dev && !S_host)) return fail(KHP_ERR_INVALID_ARG, "Y, G or S is NULL");
    if (m < 1 || m > KHP_MAX_M) return fail(KHP_ERR_INVALID_ARG, "m out of range 1..64");
    if (method < 0 || method > 2) return fail(KHP_ERR_INVALID_ARG, "method must be 0, 1 or 2");
    if (method != 1 && !oz_supported(m, m)) return fail(KHP_ERR_INVALID_ARG, "methods 0 and 2 take m <= 32");
    CKS(ensure_partial(g));
    const int nblk = std::min(dense_blocks(rows), dense_blocks(g->n));
    const double2* Y = (const double2*)Y_dev;
    const double2* W = (const double2*)W_dev;
    CK(cudaMemsetAsync(g->dflag, 0, sizeof(int), g->stream));
    if (method == 0) CK(launch_gram_tc(Y, W, rows, m, 0, m, g->partial, nblk, g->small, g->dflag, g->stream));
    else if (method == 2) CK(launch_gram_oz(Y, W, rows, m, 0, m, g->partial, nblk, g->small, g->stream));
    else CK(launch_gram(Y, W, rows, m, 0, m, g->partial, nblk, g->small, g->stream));
    CK(cudaMemcpyAsync(G_host, g->small, sizeof(double2) * m * m, cudaMemcpyDeviceToHost, g->stream));
    if (W)
        CK(cudaMemcpyAsync(S_host, g->small + m * m, sizeof(double2) * m * m, cudaMemcpyDeviceToHost, g->stream));
    int flag = 0;
    CK(cudaMemcpyAsync(&flag, g->dflag, sizeof(int), cudaMemcpyDeviceToHost, g->stream));
    CK(cudaStreamSynchronize(g->stream));
    if (flag & 8) return fail(KHP_ERR_CUDA, "tensor-core pipeline wait ran out");
    return KHP_OK;
}

khp_status khp_project(khp_handle g, const void* Y_dev, const void* W_dev, int m, int method, double* G_host,
                       double* S_host) {
    if (!g) return fail(KHP_ERR_INVALID_ARG, "handle is NULL");
    return khp_project_rows(g, Y_dev, W_dev, g->n, m, method, G_host, S_host);
}

khp_status khp_rotate(khp_handle g, const void* Y_dev, const void* W_dev, const double* Q_host, int m, int method,
                      void* X_dev, void* HX_dev) {
    g_err.clear();
    if (!g) return fail(KHP_ERR_INVALID_ARG, "handle is NULL");
    if (!Y_dev || !Q_host || !X_dev || (W_dev && !HX_dev)) return fail(KHP_ERR_INVALID_ARG, "Y, Q, X or HX is NULL");
    if (m < 1 || m > KHP_MAX_M) return fail(KHP_ERR_INVALID_ARG, "m out of range 1..64");
    if (method < 0 || method > 2) return fail(KHP_ERR_INVALID_ARG, "method must be 0, 1 or 2");
    if (method != 1 && !oz_supported(m, m)) return fail(KHP_ERR_INVALID_ARG, "methods 0 and 2 take m <= 32");
    CKS(ensure_partial(g));
    const int nblk = dense_blocks(g->n);
    double2* Qd = g->small + 2 * m * m;
    CK(cudaMemcpyAsync(Qd, Q_host, sizeof(double2) * m * m, cudaMemcpyHostToDevice, g->stream));
    const double2* Y = (const double2*)Y_dev;
    const double2* W = (const double2*)W_dev;
    CK(cudaMemsetAsync(g->dflag, 0, sizeof(int), g->stream));
    if (method == 0)
        CK(launch_rotate_tc(Y, W, m, 0, m, Qd, m, nullptr, (double2*)X_dev, (double2*)HX_dev, g->n, nullptr, nblk,
                            nullptr, g->dflag, g->stream));
    else if (method == 2)
        CK(launch_rotate_oz(Y, W, m, 0, m, Qd, m, nullptr, (double2*)X_dev, (double2*)HX_dev, g->n, nullptr, nblk,
                            nullptr, g->stream));
    else
        CK(launch_rotate(Y, W, m, 0, m, Qd, m, nullptr, (double2*)X_dev, (double2*)HX_dev, g->n, nullptr, nblk,
                         nullptr, g->stream));
    int flag = 0;
    CK(cudaMemcpyAsync(&flag, g->dflag, sizeof(int), cudaMemcpyDeviceToHost, g->stream));
    CK(cudaStreamSynchronize(g->stream));
    if (flag & 8) return fail(KHP_ERR_CUDA, "tensor-core pipeline wait ran out");
    return KHP_OK;
}

}  // extern "C"

// ============================================================ eigensolver
namespace {

struct Solver {
    khp_grid* g;
    int m;
    int nblk;
    int proj = 1;    // Gram and rotation: 0 tcgen05, 1 FP64 ALU, 2 mma.sync (split-digit, FP64 accurate)
    double2* G;      // [2 m m]: G then S
    double2* Q;      // [m m]
    double* theta;   // [m]
    double* res;     // [m]

    bool timing = false;   // record the phase events (not under stream capture)
    bool rr_timed = false;
    khp_status rr(double2* Y, double2* W) {
        if (timing) CK(cudaEventRecord(g->evp[0], g->stream));
        if (proj == 0) CK(launch_gram_tc(Y, W, g->n, m, 0, m, g->partial, nblk, G, g->dflag, g->stream));
        else if (proj == 2) CK(launch_gram_oz(Y, W, g->n, m, 0, m, g->partial, nblk, G, g->stream));
        else CK(launch_gram(Y, W, g->n, m, 0, m, g->partial, nblk, G, g->stream));
        if (timing) CK(cudaEventRecord(g->evp[1], g->stream));
        CK(launch_small(G, G + m * m, m, 1, Q, theta, g->dflag, g->stream));
        if (timing) CK(cudaEventRecord(g->evp[2], g->stream));
        if (proj == 0)
            CK(launch_rotate_tc(Y, W, m, 0, m, Q, m, theta, Y, W, g->n, (double*)g->partial, nblk, res, g->dflag,
                                g->stream));
        else if (proj == 2)
            CK(launch_rotate_oz(Y, W, m, 0, m, Q, m, theta, Y, W, g->n, (double*)g->partial, nblk, res, g->stream));
        else
            CK(launch_rotate(Y, W, m, 0, m, Q, m, theta, Y, W, g->n, (double*)g->partial, nblk, res, g->stream));
        if (timing) CK(cudaEventRecord(g->evp[3], g->stream));
        rr_timed = timing;
        g->launches += 5;
        return KHP_OK;
    }
    khp_status orth(double2* Y) {
        if (proj == 0) CK(launch_gram_tc(Y, nullptr, g->n, m, 0, m, g->partial, nblk, G, g->dflag, g->stream));
        else if (proj == 2) CK(launch_gram_oz(Y, nullptr, g->n, m, 0, m, g->partial, nblk, G, g->stream));
        else CK(launch_gram(Y, nullptr, g->n, m, 0, m, g->partial, nblk, G, g->stream));
        CK(launch_small(G, nullptr, m, 0, Q, nullptr, g->dflag, g->stream));
        if (proj == 0)
            CK(launch_rotate_tc(Y, nullptr, m, 0, m, Q, m, nullptr, Y, nullptr, g->n, nullptr, nblk, nullptr, g->dflag,
                                g->stream));
        else if (proj == 2)
            CK(launch_rotate_oz(Y, nullptr, m, 0, m, Q, m, nullptr, Y, nullptr, g->n, nullptr, nblk, nullptr, g->stream));
        else
            CK(launch_rotate(Y, nullptr, m, 0, m, Q, m, nullptr, Y, nullptr, g->n, nullptr, nblk, nullptr, g->stream));
        g->launches += 4;
        return KHP_OK;
    }
    // copies of theta, residuals and flags into pinned memory (async)
    khp_status copy_out() {
        double* hp = g->host_pinned;
        CK(cudaMemcpyAsync(hp, theta, sizeof(double) * m, cudaMemcpyDeviceToHost, g->stream));
        CK(cudaMemcpyAsync(hp + m, res, sizeof(double) * m, cudaMemcpyDeviceToHost, g->stream));
        CK(cudaMemcpyAsync(hp + 2 * m, g->dflag, sizeof(int), cudaMemcpyDeviceToHost, g->stream));
        return KHP_OK;
    }
    // after the stream is synchronised
    void read_out(std::vector<double>& th, std::vector<double>& rs, int& flags) const {
        const double* hp = g->host_pinned;
        th.assign(hp, hp + m);
        rs.assign(hp + m, hp + 2 * m);
        std::memcpy(&flags, hp + 2 * m, sizeof(int));
    }
    template <typename R>
    khp_status filter(cx_t<R>* buf[3], int& out_idx, int deg, double a, double b, double low, int c0, int nc) {
        // Y1 = (sigma1/e)(H - c)X ; Y_{k+1} = (2 s_{k+1}/e)(H - c)Y_k - s_k s_{k+1} Y_{k-1}
        const double e = 0.5 * (b - a), c = 0.5 * (b + a);
        const double sigma1 = e / (low - c);
        double sigma = sigma1;
        const double tau = 2.0 / sigma1;
        int ix = 0, iy = 1, iz = 2;
        CKS(apply_op<R>(g, buf[ix], nullptr, buf[iy], m, c0, nc, sigma1 / e, -c * sigma1 / e, 0.0));
        for (int k = 2; k <= deg; ++k) {
            const double sn = 1.0 / (tau - sigma);
            CKS(apply_op<R>(g, buf[iy], buf[ix], buf[iz], m, c0, nc, 2.0 * sn / e, -2.0 * c * sn / e, -sigma * sn));
            const int t = ix; ix = iy; iy = iz; iz = t;
            sigma = sn;
        }
        out_idx = iy;
        return KHP_OK;
    }
};

}  // namespace

namespace {

// One eigensolve as a resumable state machine, so that a single call and
// the batched call drive the same code:
//   begin()  -> [sync] absorb() -> loop { decide(); issue(); [sync] absorb(); } -> end()
// decide() takes the host decisions (convergence, phase, locking, filter
// interval and degree); issue() only enqueues device work on the handle's
// stream (it may be captured into a CUDA graph); absorb() reads back the Ritz
// values, residuals and flags that issue() copied to pinned memory.
struct Solve {
    khp_grid* g = nullptr;
    khp_solver_opts o{};
    Solver S;
    int n = 0, m = 0;
    bool mixed = false;
    int max_iter = 0;
    double tol = 0, lam_up = 0;
    int ib[4] = {0, 1, 2, 3};      // ib[0] = X (current Ritz vectors), ib[3] = W = H X
    std::vector<double> th, rs;
    int flags = 0;
    khp_stats st{};
    enum { P_FP32, P_CLEAN, P_FP64, P_DC };
    int phase = P_FP64, clean_sweeps = 0, clean_done = 0, stall = 0;
    double best = 1e300, floor32 = 0;
    bool converged = false, finished = false, timing = true, trace = false, trace_cols = false, dc = false;
    bool timed32 = false, timed64 = false, recover = false, need_bound = false;
    int it = 0;
    // decisions for the next issue()
    int nlock = 0, na = 0, deg = 0;
    double a = 0, low = 0;
    std::chrono::steady_clock::time_point t0;

    static khp_status validate(khp_grid* g, const khp_solver_opts* opts) {
        if (!g || !opts) return fail(KHP_ERR_INVALID_ARG, "handle or opts is NULL");
        if (!g->fields_set) return fail(KHP_ERR_STATE, "fields not set");
        const int n = opts->n_states, m = opts->block_m;
        if (m < 2 || m > KHP_MAX_M || (m & 1)) return fail(KHP_ERR_INVALID_ARG, "block_m must be even, 2..64");
        if (n < 1 || n >= m) return fail(KHP_ERR_INVALID_ARG, "need 1 <= n_states < block_m");
        if ((long long)m > g->n) return fail(KHP_ERR_INVALID_ARG, "block_m exceeds the number of unknowns");
        if (opts->degree < 1) return fail(KHP_ERR_INVALID_ARG, "degree must be >= 1");
        if (opts->precision < 0 || opts->precision > 2)
            return fail(KHP_ERR_INVALID_ARG, "precision must be 0, 1 or 2");
        if (!(opts->tol_ev > 0.0)) return fail(KHP_ERR_INVALID_ARG, "tol_ev must be > 0");
        if (opts->warm_start_dev && (opts->warm_cols < 1 || opts->warm_cols > m))
            return fail(KHP_ERR_INVALID_ARG, "warm_cols must be in 1..block_m");
        if (opts->start < 0 || opts->start > 1)
            return fail(KHP_ERR_INVALID_ARG, "start must be 0 (random) or 1 (coarse grid)");
        if (opts->projections < 0 || opts->projections > 2)
            return fail(KHP_ERR_INVALID_ARG,
                        "projections must be 0 (tcgen05 tensor cores), 1 (FP64 ALU) or 2 (mma.sync tensor cores)");
        return KHP_OK;
    }

    // stage a: workspace and (when the fields changed) the Lanczos bound,
    // issued on the handle's stream; the caller synchronises before begin_b
    khp_status begin_a(khp_grid* grid, const khp_solver_opts* opts) {
        t0 = std::chrono::steady_clock::now();
        g = grid;
        o = *opts;
        n = o.n_states;
        m = o.block_m;
        mixed = o.precision == 1;
        dc = o.precision == 2;
        CKS(ensure_ws(g, m, mixed || dc));
        g->launches = 0;
        need_bound = !g->bound_valid;
        if (need_bound) CKS(lanczos_issue(g, (int)std::min<long long>(40, g->n), o.seed));
        return KHP_OK;
    }

    // Coarse-grid start: the lowest m states of the 2x coarser grid (a loose
    // solve, see below), prolongated trilinearly into all m columns of X.  `started` stays false (random
    // start) when the coarse grid is too small for that block.
    khp_status coarse_start(double2* X, bool& started) {
        started = false;
        const khp_solver_opts oc = coarse_opts(o, m);
        if (!coarse_eligible(g, m, oc.block_m - m)) return KHP_OK;
        const auto tc0 = std::chrono::steady_clock::now();
        CKS(coarse_prepare(g));
        khp_grid* gc = g->coarse;
        gc->stream = g->stream;
        CKS(coarse_block(g, m));
        std::vector<double> ev(m);
        khp_stats sc_st{};
        {
            Solve sc;
            sc.timing = false;
            CKS(sc.begin_a(gc, &oc));
            CK(cudaStreamSynchronize(gc->stream));
            CKS(sc.begin_b());
            CK(cudaStreamSynchronize(gc->stream));
            CKS(sc.absorb());
            for (;;) {
                CKS(sc.decide());
                if (sc.finished) break;
                CKS(sc.issue());
                CK(cudaStreamSynchronize(gc->stream));
                CKS(sc.absorb());
            }
            const khp_status es = sc.end(ev.data(), g->coarse_x, nullptr, &sc_st);
            if (es != KHP_OK && es != KHP_ERR_NOT_CONVERGED) return es;
            g_err.clear();
        }
        CK(launch_prolong(gc, g->coarse_x, m, g, X, m, m));
        g->launches += 1 + sc_st.kernel_launches;
        st.start_iterations = sc_st.iterations;
        st.ms_start = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - tc0).count();
        started = true;
        return KHP_OK;
    }

    // set by the batched solver when it has filled the start block from the
    // coarse grids (begin_b then keeps it); its coarse statistics
    bool prefilled = false;
    int pre_iterations = 0;
    double pre_ms = 0.0;

    // stage b: random / warm start, orthonormalisation and the first
    // Rayleigh-Ritz, issued; the caller synchronises before absorb
    khp_status begin_b() {
        if (need_bound) {
            lanczos_finish(g, &g->lambda_lanczos, &g->lambda_low);
            g->bound_valid = true;
        }
        S.g = g; S.m = m; S.nblk = dense_blocks(g->n);
        S.proj = (o.projections != 1 && tc_supported(m, m)) ? o.projections : 1;
        S.G = g->small; S.Q = g->small + 2 * m * m;
        S.theta = g->dvec; S.res = g->dvec + m;
        max_iter = o.max_iter > 0 ? o.max_iter : 1000;
        tol = o.tol_ev;
        lam_up = g->lambda_lanczos;
        st = khp_stats{};
        st.lambda_upper = lam_up;
        phase = mixed ? P_FP32 : (dc ? P_DC : P_FP64);
        clean_sweeps = mixed ? (o.refine_sweeps < 0 ? 1 : o.refine_sweeps) : 0;
        // residual floor of FP32 blocks (measured on B300: ~2.5e-7 x lambda_max)
        floor32 = 3e-7 * lam_up;
        // KHP_TRACE=1 in the environment prints one line per outer iteration,
        // KHP_TRACE=2 adds the Ritz values and residuals of every column
        const char* tr = std::getenv("KHP_TRACE");
        trace = tr && (tr[0] == '1' || tr[0] == '2');
        trace_cols = tr && tr[0] == '2';
        double2** B = g->blk64;
        CK(cudaMemsetAsync(g->dflag, 0, sizeof(int) * 8, g->stream));
        bool started = prefilled;
        if (prefilled) {
            st.start_iterations = pre_iterations;
            st.ms_start = pre_ms;
        } else if (o.start == 1 && !o.warm_start_dev) {
            CKS(coarse_start(B[ib[0]], started));
        }
        if (!started) {
            CK(launch_random_fill(B[ib[0]], g->n, m, 0, m, o.seed, g->mask, g->stream, g->nb));
            g->launches += 1;
        }
        if (o.warm_start_dev)
            CK(cudaMemcpy2DAsync(B[ib[0]], sizeof(double2) * m, o.warm_start_dev, sizeof(double2) * o.warm_cols,
                                 sizeof(double2) * o.warm_cols, g->n, cudaMemcpyDeviceToDevice, g->stream));
        CKS(S.orth(B[ib[0]]));
        CKS(apply_op<double>(g, B[ib[0]], nullptr, B[ib[3]], m, 0, m, 1.0, 0.0, 0.0));
        S.timing = timing;
        CKS(S.rr(B[ib[0]], B[ib[3]]));
        CKS(S.copy_out());
        return KHP_OK;
    }

    // after the stream has been synchronised
    khp_status absorb() {
        S.read_out(th, rs, flags);
        if (timed32 || timed64) {
            float ms = 0.f;
            CK(cudaEventElapsedTime(&ms, g->ev0, g->ev1));
            if (timed32) st.ms_filter_fp32 += ms;
            else st.ms_filter_fp64 += ms;
        }
        if (S.rr_timed) {
            float t01 = 0.f, t12 = 0.f, t23 = 0.f, tf = 0.f;
            CK(cudaEventElapsedTime(&t01, g->evp[0], g->evp[1]));
            CK(cudaEventElapsedTime(&t12, g->evp[1], g->evp[2]));
            CK(cudaEventElapsedTime(&t23, g->evp[2], g->evp[3]));
            st.ms_gram += t01;
            st.ms_small += t12;
            st.ms_rotate += t23;
            // Gram: Y and W read; rotation: Y and W read, X and HX written
            st.bytes_rr += 6.0 * (double)g->n * m * sizeof(double2);
            if (timed32 || timed64) {
                CK(cudaEventElapsedTime(&tf, g->ev1, g->evp[0]));
                st.ms_between += tf;
            }
            S.rr_timed = false;
        }
        if (timed32) st.pv_fp32 += (double)g->np * na * (phase == P_DC ? deg - 1 : deg);
        if (timed64) st.pv_fp64 += (double)g->np * na * deg;
        timed32 = timed64 = false;
        {
            double rm = 0;
            for (int i = 0; i < n; ++i) rm = std::max(rm, rs[i]);
            if (st.n_history < KHP_STATS_HISTORY) st.res_history[st.n_history] = rm;
            st.n_history++;
        }
        if (trace && it > 0) {
            double rm = 0;
            for (int i = 0; i < n; ++i) rm = std::max(rm, rs[i]);
            const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
            std::fprintf(stderr, "khp it %d phase %d nlock %d deg %d a %.6e low %.6e rmax %.3e t %.1f ms\n", it - 1,
                         phase, nlock, deg, a, low, rm, ms);
        }
        if (trace_cols) {
            for (int i = 0; i < m; ++i)
                std::fprintf(stderr, "khp col it %d %d theta %.17e res %.3e\n", it, i, th[i], rs[i]);
        }
        return KHP_OK;
    }

    // host decisions; sets finished when the solve is over
    khp_status decide() {
        recover = false;
        if (flags & 8) return fail(KHP_ERR_CUDA, "stencil copy or tensor-core pipeline wait ran out");
        if (flags & 4) return fail(KHP_ERR_BREAKDOWN, "non-finite Ritz values");
        double rmax = 0;
        for (int i = 0; i < n; ++i) rmax = std::max(rmax, std::isnan(rs[i]) ? HUGE_VAL : rs[i]);
        if (rmax == HUGE_VAL) return fail(KHP_ERR_BREAKDOWN, "non-finite residuals");
        if (rmax <= tol) { converged = finished = true; return KHP_OK; }
        if (it >= max_iter) { finished = true; return KHP_OK; }
        if (phase == P_FP32) {
            // leave the FP32 phase at its floor, or when the residual stops
            // falling (two iterations without a 30 % gain below 1e-3 eV)
            if (rmax < 0.7 * best) { best = rmax; stall = 0; }
            else if (rmax < 1e-3) ++stall;
            if (rmax <= std::max(tol, floor32) || stall >= 2) {
                if (o.refine_sweeps == 0) { finished = true; return KHP_OK; }
                phase = P_CLEAN;
            }
        }
        if (phase == P_CLEAN && clean_done >= clean_sweeps) {
            if (o.refine_sweeps >= 0) { finished = true; return KHP_OK; }
            phase = P_FP64;
        }
        if (flags & 2) {
            recover = true;   // Cholesky breakdown: re-orthonormalise and redo RR
            return KHP_OK;
        }
        st.shifted_cholesky += (flags & 1) ? 1 : 0;

        // soft locking: the leading converged Ritz vectors are not filtered
        // (they stay in the Rayleigh-Ritz block with their H x)
        nlock = 0;
        while (nlock < n && rs[nlock] <= tol) ++nlock;
        nlock &= ~1;
        na = m - nlock;

        // filter interval [a, b] and scaling point low; the clean-up sweeps
        // damp everything above a point just inside the unwanted spectrum
        a = th[m - 1];
        deg = o.degree;
        if (phase == P_CLEAN) {
            a = a + 0.005 * (lam_up - a);
            deg *= 2;
        } else if (phase == P_FP32) {
            deg *= 2;   // cheap FP32 applies: fewer FP64 projections per apply
        }
        if (!(a < lam_up)) a = lam_up - 1e-3 * std::fabs(lam_up);
        // scaling point: the lower spectral estimate (or the smallest Ritz
        // value once that is lower); the degree is capped so that the
        // amplification at the bottom of the spectrum stays <= 1e4 (filtered
        // block well conditioned, no FP32 overflow; 1e5 for precision 2)
        const double lo_est = std::min(th[0], g->lambda_low);
        low = (lo_est < a) ? lo_est : a - 1e-3 * (lam_up - a);
        const double e = 0.5 * (lam_up - a), c = 0.5 * (lam_up + a);
        const double xl = std::fabs((low - c) / e);
        if (xl > 1.0) {
            // the defect-corrected mode filters the correction Z in FP32, not
            // the amplified block itself, and takes a 1e5 cap (measured at
            // C2: 7 instead of 8 outer iterations, 3 % faster)
            double cap = dc ? 1e5 : 1e4;
            // KHP_AMP_CAP in the environment overrides the cap (tuning)
            if (const char* ac = std::getenv("KHP_AMP_CAP")) {
                const double v = std::atof(ac);
                if (v > 1.0 && std::isfinite(v)) cap = v;
            }
            const int dmax = (int)std::floor(std::acosh(cap) / std::acosh(xl));
            deg = std::max(1, std::min(deg, dmax));
        }
        return KHP_OK;
    }

    // enqueue one outer iteration (no host synchronisation)
    khp_status issue() {
        double2** B = g->blk64;
        CK(cudaMemsetAsync(g->dflag, 0, sizeof(int), g->stream));
        if (recover) {
            CKS(S.orth(B[ib[0]]));
            CKS(S.orth(B[ib[0]]));
            CKS(apply_op<double>(g, B[ib[0]], nullptr, B[ib[3]], m, 0, m, 1.0, 0.0, 0.0));
            CKS(S.rr(B[ib[0]], B[ib[3]]));
            CKS(S.copy_out());
            return KHP_OK;
        }
        double2* Y = nullptr;
        if (phase == P_DC) {
            CKS(issue_dc());
            if (deferred) return KHP_OK;   // the caller launches the steps, then finish_issue()
            Y = B[ib[0]];
        } else if (phase == P_FP32) {
            float2* fb[3] = {g->blk32[0], g->blk32[1], g->blk32[2]};
            CK(launch_convert_d2f(B[ib[0]], fb[0], g->n, m, nlock, na, g->stream));
            int oi = 0;
            if (timing) CK(cudaEventRecord(g->ev0, g->stream));
            CKS(S.filter<float>(fb, oi, deg, a, lam_up, low, nlock, na));
            if (timing) CK(cudaEventRecord(g->ev1, g->stream));
            timed32 = true;
            st.launches_fp32 += deg;
            // H Y in FP32 into a free FP32 buffer, both back to FP64
            const int fw = (oi + 1) % 3;
            CKS(apply_op<float>(g, fb[oi], nullptr, fb[fw], m, nlock, na, 1.0, 0.0, 0.0));
            Y = B[ib[0]];
            CK(launch_convert_f2d(fb[oi], Y, g->n, m, nlock, na, g->stream));
            CK(launch_convert_f2d(fb[fw], B[ib[3]], g->n, m, nlock, na, g->stream));
            g->launches += 3;
            st.iterations_fp32++;
        } else {
            double2* fb[3] = {B[ib[0]], B[ib[1]], B[ib[2]]};
            int oi = 0;
            if (timing) CK(cudaEventRecord(g->ev0, g->stream));
            CKS(S.filter<double>(fb, oi, deg, a, lam_up, low, nlock, na));
            if (timing) CK(cudaEventRecord(g->ev1, g->stream));
            timed64 = true;
            st.launches_fp64 += deg;
            if (oi != 0 && nlock > 0)
                CK(cudaMemcpy2DAsync(fb[oi], sizeof(double2) * m, fb[0], sizeof(double2) * m,
                                     sizeof(double2) * nlock, g->n, cudaMemcpyDeviceToDevice, g->stream));
            // new roles: the filter output becomes X after the RR
            const int bo = ib[oi];
            int others[2], k = 0;
            for (int j = 0; j < 3; ++j)
                if (j != oi) others[k++] = ib[j];
            ib[0] = bo; ib[1] = others[0]; ib[2] = others[1];
            Y = B[ib[0]];
            CKS(apply_op<double>(g, Y, nullptr, B[ib[3]], m, nlock, na, 1.0, 0.0, 0.0));
            if (phase == P_CLEAN) clean_done++;
        }
        return issue_tail(Y);
    }

    // after the filter: Rayleigh-Ritz of Y (W = H Y in B[ib[3]]), copies out
    khp_status issue_tail(double2* Y) {
        double2** B = g->blk64;
        st.filter_applies += (long long)(deg + 1) * na / m;
        S.timing = timing;
        CKS(S.rr(Y, B[ib[3]]));
        CKS(S.copy_out());
        if (!timing) timed32 = timed64 = false;
        ++it;
        return KHP_OK;
    }

    // batched rounds: with `defer` set, issue() of a defect-corrected
    // iteration enqueues the work before the FP32 filter and hands the
    // filter's steps to the caller (one grouped launch per step across the
    // problems of the round); finish_issue() then enqueues the rest
    std::vector<StencilArgs<float>>* defer = nullptr;
    bool deferred = false;
    std::vector<double> dc_D;
    int dc_iz = 0;

    khp_status finish_issue() {
        deferred = false;
        CKS(issue_dc_tail());
        return issue_tail(g->blk64[ib[0]]);
    }

    // Defect-corrected FP32 filter: Y = X diag(D_d) + Z_d with the scalar
    // Chebyshev recurrence D_k at the Ritz values (FP64, host) and the
    // correction Z_k driven by the FP64 residual R = HX - X Theta (FP32 on
    // the device).  The d - 1 filter applies are FP32; the FP32 rounding acts
    // on Z, which shrinks with the residual.  W = H Y is one FP64 apply.
    khp_status issue_dc() {
        double2** B = g->blk64;
        float2* R32 = g->blk32[3];
        float2* zb[3] = {g->blk32[0], g->blk32[1], g->blk32[2]};
        const double e = 0.5 * (lam_up - a), cm = 0.5 * (lam_up + a);
        const double sigma1 = e / (low - cm);
        const double tau = 2.0 / sigma1;
        std::vector<double> Dprev(m, 1.0), Dcur(m, 1.0), Dnext(m, 1.0);
        for (int c = nlock; c < m; ++c) Dcur[c] = (sigma1 / e) * (th[c] - cm);
        CK(launch_dc_residual(B[ib[0]], B[ib[3]], R32, zb[0], g->n, m, nlock, na, th.data(), sigma1 / e,
                              g->stream));
        g->launches += 1;
        if (timing && !defer) CK(cudaEventRecord(g->ev0, g->stream));
        int iz = 0, ip = -1, in = 1;
        double sigma = sigma1;
        for (int k = 1; k < deg; ++k) {
            const double sn = 1.0 / (tau - sigma);
            const double al = 2.0 * sn / e, be = -2.0 * cm * sn / e, ga = -sigma * sn;
            StencilArgs<float> sa;
            sa.nx = g->nx; sa.ny = g->ny; sa.nz = g->nz;
            sa.ld = m; sa.col0 = nlock; sa.ncol = na;
            sa.alpha = (float)al; sa.beta = (float)be; sa.gamma = (float)ga;
            sa.x = zb[iz]; sa.prev = ip >= 0 ? zb[ip] : nullptr; sa.y = zb[in];
            sa.onsite = g->onsite32;
            sa.phase = (const float2*)(g->has_phase ? g->phase32 : nullptr);
            sa.phase_mode = g->has_phase ? g->phase_mode : PH_NONE;
            sa.mask = g->mask;
            sa.src = R32;
            sa.nb = g->nb;
            sa.err = g->dflag;
            for (int c = 0; c < 64; ++c) sa.src_coef[c] = (c >= nlock && c < m) ? (float)(al * Dcur[c]) : 0.f;
            fill_coeffs<float>(g, sa.c, al);
            if (defer) defer->push_back(sa);
            else CK(launch_stencil<float>(sa, g->stream));
            g->launches += 1;
            for (int c = nlock; c < m; ++c) Dnext[c] = al * (th[c] - cm) * Dcur[c] + ga * Dprev[c];
            std::swap(Dprev, Dcur);
            std::swap(Dcur, Dnext);
            const int free_ = (ip >= 0) ? ip : 3 - iz - in;
            ip = iz; iz = in; in = free_;
            sigma = sn;
        }
        st.launches_fp32 += deg - 1;
        dc_D = Dcur;
        dc_iz = iz;
        if (defer) {
            // the steps run in the caller's grouped launches: no filter timing
            deferred = true;
            timed32 = false;
            return KHP_OK;
        }
        if (timing) CK(cudaEventRecord(g->ev1, g->stream));
        timed32 = true;
        return issue_dc_tail();
    }

    // Y = X D + Z in FP64, then W = H Y (FP64) on the active columns
    khp_status issue_dc_tail() {
        double2** B = g->blk64;
        float2* zb[3] = {g->blk32[0], g->blk32[1], g->blk32[2]};
        CK(launch_dc_combine(B[ib[0]], B[ib[3]], zb[dc_iz], B[ib[1]], B[ib[2]], g->n, m, nlock, dc_D.data(),
                             g->stream));
        g->launches += 1;
        CKS(apply_op<double>(g, B[ib[1]], nullptr, B[ib[2]], m, nlock, na, 1.0, 0.0, 0.0));
        // roles: Y, W become the next X, HX after the Rayleigh-Ritz
        const int x0 = ib[0], w0 = ib[3];
        ib[0] = ib[1];
        ib[3] = ib[2];
        ib[1] = x0;
        ib[2] = w0;
        return KHP_OK;
    }

    khp_status end(double* evals_host, void* evecs_dev, double* resid_host, khp_stats* stats) {
        double2** B = g->blk64;
        // final orthonormalisation of the Ritz block
        CKS(S.orth(B[ib[0]]));
        CK(cudaMemcpy2DAsync(evecs_dev, sizeof(double2) * n, B[ib[0]], sizeof(double2) * m, sizeof(double2) * n,
                             g->n, cudaMemcpyDeviceToDevice, g->stream));
        if (o.block_out_dev)
            CK(cudaMemcpyAsync(o.block_out_dev, B[ib[0]], sizeof(double2) * g->n * m, cudaMemcpyDeviceToDevice,
                               g->stream));
        CK(cudaStreamSynchronize(g->stream));
        for (int i = 0; i < n; ++i) evals_host[i] = th[i];
        double rmax = 0;
        int conv = 0;
        for (int i = 0; i < n; ++i) {
            rmax = std::max(rmax, rs[i]);
            conv += rs[i] <= tol;
            if (resid_host) resid_host[i] = rs[i];
        }
        st.iterations = it;
        st.block_m = m;
        st.converged = conv;
        st.kernel_launches = g->launches;
        st.point_vectors = (double)g->np * m;
        op_counts(g, m, &st.flops_per_pv, &st.bytes_per_pv_fp64, &st.bytes_per_pv_fp32);
        st.max_residual = rmax;
        st.ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        if (stats) *stats = st;
        if (!converged && !(mixed && o.refine_sweeps >= 0 && it < max_iter))
            return fail(KHP_ERR_NOT_CONVERGED, "max_iter reached before all residuals <= tol_ev");
        return KHP_OK;
    }
};

}  // namespace

extern "C" khp_status khp_eigensolve(khp_handle g, const khp_solver_opts* opts, double* evals_host,
                                     void* evecs_dev, double* resid_host, khp_stats* stats) {
    g_err.clear();
    CKS(Solve::validate(g, opts));
    if (!evals_host || !evecs_dev) return fail(KHP_ERR_INVALID_ARG, "evals or evecs is NULL");
    Solve s;
    CKS(s.begin_a(g, opts));
    CK(cudaStreamSynchronize(g->stream));
    CKS(s.begin_b());
    CK(cudaStreamSynchronize(g->stream));
    CKS(s.absorb());
    for (;;) {
        CKS(s.decide());
        if (s.finished) break;
        CKS(s.issue());
        CK(cudaStreamSynchronize(g->stream));
        CKS(s.absorb());
    }
    return s.end(evals_host, evecs_dev, resid_host, stats);
}


// ------------------------------------------------------------- batched
namespace {

// Streams of a batch: every handle gets its own non-blocking stream for the
// call (ordered after the handle's own stream on entry and before it on
// exit), so the problems' kernels can overlap and the rounds can be captured.
struct BatchStreams {
    std::vector<khp_grid*> gs;
    std::vector<cudaStream_t> orig, own;
    std::vector<cudaEvent_t> ev;
    cudaStream_t master = nullptr;
    ~BatchStreams() {
        for (size_t i = 0; i < gs.size(); ++i) {
            if (own[i]) {
                cudaEventRecord(ev[i], own[i]);
                cudaStreamWaitEvent(orig[i], ev[i], 0);
                gs[i]->stream = orig[i];
                cudaStreamDestroy(own[i]);
            }
            if (ev[i]) cudaEventDestroy(ev[i]);
        }
        if (master) cudaStreamDestroy(master);
    }
};

}  // namespace

extern "C" khp_status khp_eigensolve_batched(const khp_handle* hs, int count, const khp_solver_opts* opts,
                                             double* evals_host, void* const* evecs_dev, double* resid_host,
                                             khp_stats* stats, int flags) {
    g_err.clear();
    if (!hs || !opts || !evals_host || !evecs_dev) return fail(KHP_ERR_INVALID_ARG, "NULL argument");
    if (count < 1) return fail(KHP_ERR_INVALID_ARG, "count must be >= 1");
    if (opts->warm_start_dev) return fail(KHP_ERR_INVALID_ARG, "warm starts are per problem: not in batched mode");
    if (opts->block_out_dev) return fail(KHP_ERR_INVALID_ARG, "block output is per problem: not in batched mode");
    khp_solver_opts o = *opts;
    const int n = o.n_states;
    int dev0 = -1;
    for (int i = 0; i < count; ++i) {
        if (!hs[i] || !evecs_dev[i]) return fail(KHP_ERR_INVALID_ARG, "NULL handle or evecs");
        if (i == 0) dev0 = hs[i]->device;
        if (hs[i]->device != dev0) return fail(KHP_ERR_INVALID_ARG, "all handles must be on one device");
        for (int j = 0; j < i; ++j)
            if (hs[j] == hs[i]) return fail(KHP_ERR_INVALID_ARG, "a handle appears twice");
        if (!hs[i]->fields_set) return fail(KHP_ERR_STATE, "fields not set");
    }
    if ((flags & KHP_BATCH_AUTOTUNE) == 0) CKS(Solve::validate(hs[0], &o));
    const bool graph = (flags & KHP_BATCH_GRAPH) != 0;

    BatchStreams bs;
    bs.gs.assign(hs, hs + count);
    bs.orig.resize(count);
    bs.own.assign(count, nullptr);
    bs.ev.assign(count, nullptr);
    for (int i = 0; i < count; ++i) {
        khp_grid* g = hs[i];
        bs.orig[i] = g->stream;
        CK(cudaEventCreateWithFlags(&bs.ev[i], cudaEventDisableTiming));
        CK(cudaStreamCreateWithFlags(&bs.own[i], cudaStreamNonBlocking));
        CK(cudaEventRecord(bs.ev[i], g->stream));
        CK(cudaStreamWaitEvent(bs.own[i], bs.ev[i], 0));
        g->stream = bs.own[i];
    }
    CK(cudaStreamCreateWithFlags(&bs.master, cudaStreamNonBlocking));

    // autotuner: block width chosen by timed trial solves of the smallest
    // problem (its best trial is kept as its answer)
    int tuned_from = -1;
    double tune_ms = 0.0;
    if (flags & KHP_BATCH_AUTOTUNE) {
        int small = 0;
        for (int i = 1; i < count; ++i)
            if (hs[i]->n < hs[small]->n) small = i;
        double best = 1e300;
        int best_m = 0;
        for (int cand = 0; cand < 3; ++cand) {
            khp_solver_opts t = o;
            t.block_m = std::min(KHP_MAX_M, ((n + 4 * (cand + 1)) + 1) & ~1);
            if (t.block_m <= n) continue;
            CKS(Solve::validate(hs[small], &t));
            const auto ta = std::chrono::steady_clock::now();
            khp_stats ts{};
            khp_status r = khp_eigensolve(hs[small], &t, evals_host + (size_t)small * n, evecs_dev[small],
                                          resid_host ? resid_host + (size_t)small * n : nullptr, &ts);
            if (r != KHP_OK && r != KHP_ERR_NOT_CONVERGED) return r;
            const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - ta).count();
            tune_ms += ms;
            if (r == KHP_OK && ms < best) {
                best = ms;
                best_m = t.block_m;
                if (stats) stats[small] = ts;
            }
        }
        if (best_m == 0) return fail(KHP_ERR_NOT_CONVERGED, "autotuner: no candidate block width converged");
        o.block_m = best_m;
        tuned_from = small;
        // the tuned problem is re-solved with the chosen width so that every
        // answer comes from the same configuration
    }
    for (int i = 0; i < count; ++i) CKS(Solve::validate(hs[i], &o));

    std::vector<Solve> S(count);
    // the set-up of all problems overlaps: Lanczos bounds, then first RR
    for (int i = 0; i < count; ++i) {
        S[i].timing = !graph;
        CKS(S[i].begin_a(hs[i], &o));
    }
    for (int i = 0; i < count; ++i) CK(cudaStreamSynchronize(hs[i]->stream));
    if (o.start == 1) {
        // coarse-grid start: the coarse grids of the eligible problems solved
        // together (one batched call), each block prolongated into its
        // problem's start block; the others start from random blocks
        const auto tc0 = std::chrono::steady_clock::now();
        const int m = o.block_m;
        const khp_solver_opts oc = coarse_opts(o, m);
        std::vector<int> ci;
        std::vector<khp_handle> hc;
        std::vector<void*> xc;
        for (int i = 0; i < count; ++i) {
            if (!coarse_eligible(hs[i], m, oc.block_m - m)) continue;
            CKS(coarse_prepare(hs[i]));
            hs[i]->coarse->stream = hs[i]->stream;
            CKS(coarse_block(hs[i], m));
            ci.push_back(i);
            hc.push_back(hs[i]->coarse);
            xc.push_back(hs[i]->coarse_x);
        }
        if (!hc.empty()) {
            std::vector<double> ev(hc.size() * (size_t)m);
            std::vector<khp_stats> cst(hc.size());
            const khp_status r = khp_eigensolve_batched(hc.data(), (int)hc.size(), &oc, ev.data(), xc.data(), nullptr,
                                                        cst.data(), flags & (KHP_BATCH_GRAPH | KHP_BATCH_GROUPED));
            if (r != KHP_OK && r != KHP_ERR_NOT_CONVERGED) return r;
            g_err.clear();
            const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - tc0).count();
            for (size_t k = 0; k < ci.size(); ++k) {
                const int i = ci[k];
                khp_grid* g = hs[i];
                CK(launch_prolong(g->coarse, g->coarse_x, m, g, g->blk64[S[i].ib[0]], m, m));
                g->launches += 1 + cst[k].kernel_launches;
                // the batch streams end with this call: the coarse handle goes
                // back to the fine handle's own stream
                g->coarse->stream = bs.orig[i];
                S[i].prefilled = true;
                S[i].pre_iterations = cst[k].iterations;
                S[i].pre_ms = ms;
            }
        }
    }
    for (int i = 0; i < count; ++i) CKS(S[i].begin_b());
    for (int i = 0; i < count; ++i) {
        CK(cudaStreamSynchronize(hs[i]->stream));
        CKS(S[i].absorb());
    }
    std::vector<cudaEvent_t> join(count, nullptr);
    cudaEvent_t fork = nullptr;
    struct EvGuard {
        std::vector<cudaEvent_t>* j; cudaEvent_t* f;
        ~EvGuard() { for (auto e : *j) if (e) cudaEventDestroy(e); if (*f) cudaEventDestroy(*f); }
    } evg{&join, &fork};
    CK(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
    for (int i = 0; i < count; ++i) CK(cudaEventCreateWithFlags(&join[i], cudaEventDisableTiming));
    cudaGraphExec_t exec = nullptr;
    struct ExecGuard { cudaGraphExec_t* e; ~ExecGuard() { if (*e) cudaGraphExecDestroy(*e); } } xg{&exec};
    int rounds = 0, graphs_built = 0;
    for (;;) {
        std::vector<int> act;
        for (int i = 0; i < count; ++i) {
            if (S[i].finished) continue;
            CKS(S[i].decide());
            if (!S[i].finished) act.push_back(i);
        }
        if (act.empty()) break;
        bool grouped = (flags & KHP_BATCH_GROUPED) != 0;
        for (int i : act) grouped = grouped && S[i].phase == Solve::P_DC && !S[i].recover;
        if (grouped) {
            // the round on the master stream: every problem's work before
            // its filter, then step k of all filters as grouped launches,
            // then every problem's combine, H Y and Rayleigh-Ritz
            for (int i : act) hs[i]->stream = bs.master;
            struct Restore {
                std::vector<int>* act; BatchStreams* bs; const khp_handle* hs;
                ~Restore() { for (int i : *act) hs[i]->stream = bs->own[i]; }
            } restore{&act, &bs, hs};
            if (graph) CK(cudaStreamBeginCapture(bs.master, cudaStreamCaptureModeThreadLocal));
            auto body = [&]() -> khp_status {
                std::vector<std::vector<StencilArgs<float>>> steps(count);
                size_t kmax = 0;
                for (int i : act) {
                    S[i].defer = &steps[i];
                    const khp_status r = S[i].issue();
                    S[i].defer = nullptr;
                    if (r != KHP_OK) return r;
                    kmax = std::max(kmax, steps[i].size());
                }
                std::vector<const StencilArgs<float>*> ptr;
                for (size_t k = 0; k < kmax; ++k) {
                    ptr.clear();
                    for (int i : act)
                        if (k < steps[i].size()) ptr.push_back(&steps[i][k]);
                    const cudaError_t e = launch_stencil_plane_group(ptr.data(), (int)ptr.size(), bs.master);
                    if (e == cudaErrorNotSupported) {
                        for (const StencilArgs<float>* a : ptr) CK(launch_stencil<float>(*a, bs.master));
                    } else {
                        CK(e);
                    }
                }
                for (int i : act)
                    if (S[i].deferred) CKS(S[i].finish_issue());
                return KHP_OK;
            };
            const khp_status bsr = body();
            if (graph) {
                cudaGraph_t gr = nullptr;
                const cudaError_t ee = cudaStreamEndCapture(bs.master, &gr);
                if (bsr != KHP_OK) { if (gr) cudaGraphDestroy(gr); return bsr; }
                if (ee != cudaSuccess) {
                    if (gr) cudaGraphDestroy(gr);
                    return fail(KHP_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(ee));
                }
                bool updated = false;
                if (exec) {
                    cudaGraphExecUpdateResultInfo info;
                    updated = cudaGraphExecUpdate(exec, gr, &info) == cudaSuccess;
                    if (!updated) {
                        cudaGetLastError();
                        cudaGraphExecDestroy(exec);
                        exec = nullptr;
                    }
                }
                if (!updated) {
                    const cudaError_t ie = cudaGraphInstantiate(&exec, gr, 0);
                    if (ie != cudaSuccess) { cudaGraphDestroy(gr); exec = nullptr; CK(ie); }
                    graphs_built++;
                }
                cudaGraphDestroy(gr);
                CK(cudaGraphLaunch(exec, bs.master));
            } else if (bsr != KHP_OK) {
                return bsr;
            }
            CK(cudaStreamSynchronize(bs.master));
        } else if (graph) {
            // one CUDA graph per round: fork every active problem's iteration
            // from the master stream onto its own stream and join back
            CK(cudaStreamBeginCapture(bs.master, cudaStreamCaptureModeThreadLocal));
            khp_status cs = KHP_OK;
            cudaError_t ce = cudaEventRecord(fork, bs.master);
            for (int i : act) {
                if (ce != cudaSuccess || cs != KHP_OK) break;
                ce = cudaStreamWaitEvent(hs[i]->stream, fork, 0);
                if (ce == cudaSuccess) cs = S[i].issue();
                if (ce == cudaSuccess && cs == KHP_OK) ce = cudaEventRecord(join[i], hs[i]->stream);
                if (ce == cudaSuccess && cs == KHP_OK) ce = cudaStreamWaitEvent(bs.master, join[i], 0);
            }
            cudaGraph_t gr = nullptr;
            const cudaError_t ee = cudaStreamEndCapture(bs.master, &gr);
            if (cs != KHP_OK) { if (gr) cudaGraphDestroy(gr); return cs; }
            if (ce != cudaSuccess || ee != cudaSuccess) {
                if (gr) cudaGraphDestroy(gr);
                return fail(KHP_ERR_CUDA, std::string("graph capture: ") +
                                              cudaGetErrorString(ce != cudaSuccess ? ce : ee));
            }
            bool updated = false;
            if (exec) {
                cudaGraphExecUpdateResultInfo info;
                updated = cudaGraphExecUpdate(exec, gr, &info) == cudaSuccess;
                if (!updated) {
                    cudaGetLastError();
                    cudaGraphExecDestroy(exec);
                    exec = nullptr;
                }
            }
            if (!updated) {
                const cudaError_t ie = cudaGraphInstantiate(&exec, gr, 0);
                if (ie != cudaSuccess) { cudaGraphDestroy(gr); exec = nullptr; CK(ie); }
                graphs_built++;
            }
            cudaGraphDestroy(gr);
            CK(cudaGraphLaunch(exec, bs.master));
            CK(cudaStreamSynchronize(bs.master));
        } else {
            for (int i : act) CKS(S[i].issue());
            for (int i : act) CK(cudaStreamSynchronize(hs[i]->stream));
        }
        for (int i : act) CKS(S[i].absorb());
        rounds++;
    }
    khp_status worst = KHP_OK;
    for (int i = 0; i < count; ++i) {
        khp_stats st{};
        const khp_status r = S[i].end(evals_host + (size_t)i * n, evecs_dev[i],
                                      resid_host ? resid_host + (size_t)i * n : nullptr, &st);
        st.batch_rounds = rounds;
        st.batch_graphs = graphs_built;
        st.autotune_ms = (i == tuned_from) ? tune_ms : 0.0;
        if (stats) stats[i] = st;
        if (r != KHP_OK && worst == KHP_OK) worst = r;
    }
    if (worst != KHP_OK) return fail(worst, "at least one problem did not converge");
    return KHP_OK;
}

extern "C" khp_status khp_pair_densities(khp_handle g, const void* evecs_dev, int n, void* rho_dev) {
    g_err.clear();
    if (!g) return fail(KHP_ERR_INVALID_ARG, "handle is NULL");
    if (!evecs_dev || !rho_dev) return fail(KHP_ERR_INVALID_ARG, "evecs or rho is NULL");
    if (n < 1 || n > KHP_MAX_M) return fail(KHP_ERR_INVALID_ARG, "n out of range 1..64");
    CK(launch_pair_density((const double2*)evecs_dev, g->np, n, g->nb, (double2*)rho_dev, g->stream));
    g->launches += 1;
    return KHP_OK;
}

extern "C" khp_status khp_position_moments(khp_handle g, const void* X_dev, int m, double* D_host) {
    g_err.clear();
    if (!g) return fail(KHP_ERR_INVALID_ARG, "handle is NULL");
    if (!X_dev || !D_host) return fail(KHP_ERR_INVALID_ARG, "X or D is NULL");
    if (m < 1 || m > KHP_MAX_MOMENT_M) return fail(KHP_ERR_INVALID_ARG, "m out of range 1..16");
    CKS(ensure_partial(g));
    CK(launch_moments((const double2*)X_dev, g->nx, g->ny, g->nz, g->nb, m, g->h, g->partial, g->partial_elems,
                      g->small, g->stream));
    g->launches += 2;
    CK(cudaMemcpyAsync(D_host, g->small, sizeof(double2) * 3 * m * m, cudaMemcpyDeviceToHost, g->stream));
    CK(cudaStreamSynchronize(g->stream));
    return KHP_OK;
}

extern "C" khp_status khp_density(khp_handle g, const void* evecs_dev, int n, const double* w_host,
                                  double* rho_dev) {
    g_err.clear();
    if (!g) return fail(KHP_ERR_INVALID_ARG, "handle is NULL");
    if (!evecs_dev || !w_host || !rho_dev) return fail(KHP_ERR_INVALID_ARG, "NULL argument");
    if (n < 1 || n > KHP_MAX_M) return fail(KHP_ERR_INVALID_ARG, "n out of range 1..64");
    if (!finite_all(w_host, n)) return fail(KHP_ERR_INVALID_ARG, "weights non-finite");
    CK(launch_density((const double2*)evecs_dev, g->np, n, w_host, g->mask, rho_dev, g->stream, g->nb));
    return KHP_OK;
}

extern "C" khp_status khp_state_densities(khp_handle g, const void* evecs_dev, int n, double* dens_dev) {
    g_err.clear();
    if (!g) return fail(KHP_ERR_INVALID_ARG, "handle is NULL");
    if (!evecs_dev || !dens_dev) return fail(KHP_ERR_INVALID_ARG, "NULL argument");
    if (n < 1 || n > KHP_MAX_M) return fail(KHP_ERR_INVALID_ARG, "n out of range 1..64");
    CK(launch_state_densities((const double2*)evecs_dev, g->np, n, g->nb, dens_dev, g->stream));
    g->launches += 1;
    return KHP_OK;
}

extern "C" khp_status khp_eigs_backward(khp_handle g, const void* evecs_dev, const double* evals_host,
                                        int n, const double* dLdE_host, double* dLdV_dev,
                                        double* dLdstrain_dev, const double* levers_dev, int n_gates,
                                        double* dLdalpha_host) {
    g_err.clear();
    if (!g) return fail(KHP_ERR_INVALID_ARG, "handle is NULL");
    if (!evecs_dev || !evals_host || !dLdE_host || !dLdV_dev) return fail(KHP_ERR_INVALID_ARG, "NULL argument");
    if (n < 1 || n > KHP_MAX_M) return fail(KHP_ERR_INVALID_ARG, "n out of range 1..64");
    if (n_gates < 0 || n_gates > KHP_MAX_GATES) return fail(KHP_ERR_INVALID_ARG, "n_gates out of range");
    if (n_gates > 0 && (!levers_dev || !dLdalpha_host)) return fail(KHP_ERR_INVALID_ARG, "levers/alpha output NULL");
    if (!finite_all(dLdE_host, n) || !finite_all(evals_host, n)) return fail(KHP_ERR_INVALID_ARG, "non-finite input");
    // dL/dE must be constant on every degenerate cluster
    for (int i = 0; i < n;) {
        int j = i + 1;
        while (j < n && evals_host[j] - evals_host[j - 1] <= 1e-6) ++j;
        for (int k = i + 1; k < j; ++k)
            if (std::fabs(dLdE_host[k] - dLdE_host[i]) > 1e-12 * std::max(1.0, std::fabs(dLdE_host[i])))
                return fail(KHP_ERR_DEGENERATE, "dL/dE differs inside a degenerate cluster");
        i = j;
    }
    const int nblk = 2 * 148;
    double* partial = nullptr;
    CK(cudaMallocAsync(&partial, sizeof(double) * nblk * std::max(1, n_gates), g->stream));
    double* dalpha = g->dvec + 6 * KHP_MAX_M;
    khp_status s = KHP_OK;
    cudaError_t e = launch_backward((const double2*)evecs_dev, g->np, n, dLdE_host, g->De, dLdV_dev,
                                    dLdstrain_dev, n_gates ? levers_dev : nullptr, n_gates, partial, nblk,
                                    dalpha, g->stream, g->nb);
    if (e == cudaSuccess && n_gates > 0) {
        e = cudaMemcpyAsync(g->host_pinned, dalpha, sizeof(double) * n_gates, cudaMemcpyDeviceToHost, g->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
        if (e == cudaSuccess)
            for (int k = 0; k < n_gates; ++k) dLdalpha_host[k] = g->host_pinned[k];
    }
    cudaFreeAsync(partial, g->stream);
    if (e != cudaSuccess) s = fail(KHP_ERR_CUDA, std::string("backward: ") + cudaGetErrorString(e));
    return s;
}
