// Dense FP64 pieces of the Chebyshev-filtered subspace iteration: the Gram
// contractions G = Y^H Y and S = Y^H (H Y) over the long grid dimension, the
// subspace rotation [Y, HY] Q with fused residual norms, and the one-CTA
// m x m kernels (equilibrated Cholesky, triangular inverse, Hermitian Jacobi
// eigensolver) that turn G and S into the Rayleigh-Ritz rotation.
//
// Reductions over the grid run in two deterministic stages: each CTA owns a
// contiguous row range and writes its partial m x m sums to a scratch array;
// a second kernel adds the partials in block order.
#include <math.h>

#include "khp_common.cuh"
#include "khp_internal.h"

namespace khp {

static constexpr int kThreads = 256;

int dense_blocks(long long rows) {
    long long b = rows / 512;
    if (b < 1) b = 1;
    if (b > 4 * 148) b = 4 * 148;
    return (int)b;
}

size_t gram_partial_elems(int m, int nblk) { return (size_t)nblk * 2 * m * m; }

// ------------------------------------------------------------------ Gram
// G = Y^H Y and S = Y^H W are Hermitian (S because W = H Y with H Hermitian),
// so only their upper triangles are accumulated (packed row by row,
// mt = m(m+1)/2 entries each); the reduction writes both triangles.
template <int K>
__global__ void __launch_bounds__(kThreads) gram_kernel(const double2* __restrict__ Y,
                                                       const double2* __restrict__ W, long long rows,
                                                       int ld, int col0, int m,
                                                       double2* __restrict__ partial) {
    constexpr int TR = 16;
    extern __shared__ double2 sm[];
    double2* Ys = sm;
    double2* Ws = sm + TR * m;
    const int tid = threadIdx.x;
    const int mt = m * (m + 1) / 2;
    const int E = (W ? 2 : 1) * mt;
    const long long per = (rows + gridDim.x - 1) / gridDim.x;
    const long long r0 = (long long)blockIdx.x * per;
    const long long r1 = r0 + per < rows ? r0 + per : rows;

    double2 acc[K];
    int ia[K], jb[K];
    bool sw[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        acc[k] = make_double2(0.0, 0.0);
        const int e = tid + k * kThreads;
        ia[k] = -1;
        jb[k] = 0;
        sw[k] = e >= mt;
        if (e < E) packed_ij(e % mt, m, ia[k], jb[k]);
    }
    for (long long rb = r0; rb < r1; rb += TR) {
        const int nr = (int)((r1 - rb) < TR ? (r1 - rb) : TR);
        for (int idx = tid; idx < TR * m; idx += kThreads) {
            const int r = idx / m, c = idx - r * m;
            const bool ok = r < nr;
            Ys[idx] = ok ? Y[(rb + r) * ld + col0 + c] : make_double2(0.0, 0.0);
            if (W) Ws[idx] = ok ? W[(rb + r) * ld + col0 + c] : make_double2(0.0, 0.0);
        }
        __syncthreads();
#pragma unroll 4
        for (int r = 0; r < TR; ++r) {
#pragma unroll
            for (int k = 0; k < K; ++k) {
                if (ia[k] >= 0) {
                    const double2 a = Ys[r * m + ia[k]];
                    const double2 b = sw[k] ? Ws[r * m + jb[k]] : Ys[r * m + jb[k]];
                    cfmac(acc[k], a, b);
                }
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const int e = tid + k * kThreads;
        if (e < E) partial[(size_t)blockIdx.x * E + e] = acc[k];
    }
}

// sums the packed partials in block order and writes the full Hermitian
// matrices: out[0 .. m*m) = G, out[m*m .. 2 m*m) = S
__global__ void sum_partials_herm(const double2* __restrict__ partial, int nblk, int m, int nmat,
                                  double2* __restrict__ out) {
    const int mt = m * (m + 1) / 2;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nmat * mt) return;
    const int E = nmat * mt;
    double2 s = make_double2(0.0, 0.0);
    for (int b = 0; b < nblk; ++b) {
        const double2 v = partial[(size_t)b * E + e];
        s.x += v.x;
        s.y += v.y;
    }
    const int which = e / mt;
    int i, j;
    packed_ij(e - which * mt, m, i, j);
    double2* o = out + (size_t)which * m * m;
    if (i == j) {
        o[i * m + i] = make_double2(s.x, 0.0);
    } else {
        o[i * m + j] = s;
        o[j * m + i] = make_double2(s.x, -s.y);
    }
}

cudaError_t launch_sum_partials_herm(const double2* partial, int nblk, int m, int nmat, double2* out,
                                     cudaStream_t st) {
    const int E = nmat * m * (m + 1) / 2;
    sum_partials_herm<<<(E + 255) / 256, 256, 0, st>>>(partial, nblk, m, nmat, out);
    return cudaGetLastError();
}

cudaError_t launch_gram(const double2* Y, const double2* W, long long rows, int ld, int col0, int m,
                        double2* partial, int nblk, double2* out, cudaStream_t st) {
    const int nmat = W ? 2 : 1;
    const int E = nmat * m * (m + 1) / 2;
    const int K = (E + kThreads - 1) / kThreads;
    const size_t smem = 2ull * 16 * m * sizeof(double2);
    if (K <= 1) gram_kernel<1><<<nblk, kThreads, smem, st>>>(Y, W, rows, ld, col0, m, partial);
    else if (K <= 2) gram_kernel<2><<<nblk, kThreads, smem, st>>>(Y, W, rows, ld, col0, m, partial);
    else if (K <= 4) gram_kernel<4><<<nblk, kThreads, smem, st>>>(Y, W, rows, ld, col0, m, partial);
    else if (K <= 8) gram_kernel<8><<<nblk, kThreads, smem, st>>>(Y, W, rows, ld, col0, m, partial);
    else gram_kernel<16><<<nblk, kThreads, smem, st>>>(Y, W, rows, ld, col0, m, partial);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    sum_partials_herm<<<(E + 255) / 256, 256, 0, st>>>(partial, nblk, m, nmat, out);
    return cudaGetLastError();
}

// --------------------------------------------------------------- rotation
__global__ void __launch_bounds__(kThreads) rotate_kernel(
    const double2* Y, const double2* W, int ld, int col0, int m,
    const double2* __restrict__ Q, int mq, const double* __restrict__ theta, double2* X,
    double2* HX, long long rows, double* __restrict__ res_partial) {
    constexpr int TR = 32;
    extern __shared__ double2 sm[];
    double2* Qs = sm;                 // [m][mq]
    double2* Ys = Qs + m * mq;        // [TR][m]
    double2* Ws = Ys + TR * m;        // [TR][m]
    __shared__ double red[2][kThreads];
    const int tid = threadIdx.x;
    for (int i = tid; i < m * mq; i += kThreads) Qs[i] = Q[i];
    const int j = tid % mq;
    const int rg = tid / mq;
    const int RG = kThreads / mq;
    const bool active = rg < RG;
    const double th = (theta && active) ? theta[j] : 0.0;
    double rs = 0.0, xs = 0.0;
    const long long per = (rows + gridDim.x - 1) / gridDim.x;
    const long long r0 = (long long)blockIdx.x * per;
    const long long r1 = r0 + per < rows ? r0 + per : rows;
    for (long long rb = r0; rb < r1; rb += TR) {
        const int nr = (int)((r1 - rb) < TR ? (r1 - rb) : TR);
        __syncthreads();
        for (int idx = tid; idx < nr * m; idx += kThreads) {
            const int r = idx / m, c = idx - r * m;
            Ys[idx] = Y[(rb + r) * ld + col0 + c];
            if (W) Ws[idx] = W[(rb + r) * ld + col0 + c];
        }
        __syncthreads();
        if (active) {
            for (int r = rg; r < nr; r += RG) {
                double2 x = make_double2(0.0, 0.0), hx = make_double2(0.0, 0.0);
                for (int i = 0; i < m; ++i) {
                    const double2 q = Qs[i * mq + j];
                    cfma(x, Ys[r * m + i], q);
                    if (W) cfma(hx, Ws[r * m + i], q);
                }
                X[(rb + r) * ld + col0 + j] = x;
                if (W) HX[(rb + r) * ld + col0 + j] = hx;
                if (theta) {
                    const double dx = hx.x - th * x.x, dy = hx.y - th * x.y;
                    rs += dx * dx + dy * dy;
                    xs += x.x * x.x + x.y * x.y;
                }
            }
        }
    }
    if (!res_partial) return;
    red[0][tid] = rs;
    red[1][tid] = xs;
    __syncthreads();
    if (tid < mq) {
        double a = 0.0, b = 0.0;
        for (int g = 0; g < RG; ++g) {
            a += red[0][g * mq + tid];
            b += red[1][g * mq + tid];
        }
        res_partial[(size_t)blockIdx.x * 2 * mq + tid] = a;
        res_partial[(size_t)blockIdx.x * 2 * mq + mq + tid] = b;
    }
}

__global__ void residual_finish(const double* __restrict__ partial, int nblk, int mq,
                                double* __restrict__ out) {
    const int j = threadIdx.x;
    if (j >= mq) return;
    double a = 0.0, b = 0.0;
    for (int k = 0; k < nblk; ++k) {
        a += partial[(size_t)k * 2 * mq + j];
        b += partial[(size_t)k * 2 * mq + mq + j];
    }
    out[j] = b > 0.0 ? sqrt(a / b) : 0.0;
}

cudaError_t launch_residual_finish(const double* partial, int nblk, int mq, double* out, cudaStream_t st) {
    residual_finish<<<1, 64, 0, st>>>(partial, nblk, mq, out);
    return cudaGetLastError();
}

cudaError_t launch_rotate(const double2* Y, const double2* W, int ld, int col0, int m,
                          const double2* Q, int mq, const double* theta, double2* X, double2* HX,
                          long long rows, double* res_partial, int nblk, double* res_out,
                          cudaStream_t st) {
    const size_t smem = ((size_t)m * mq + 2ull * 32 * m) * sizeof(double2);
    static bool attr_set = false;
    if (!attr_set) {
        cudaFuncSetAttribute(rotate_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
        attr_set = true;
    }
    const bool want_res = theta && W && res_partial && res_out;
    rotate_kernel<<<nblk, kThreads, smem, st>>>(Y, W, ld, col0, m, Q, mq, want_res ? theta : nullptr,
                                               X, HX, rows, want_res ? res_partial : nullptr);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || !want_res) return e;
    residual_finish<<<1, 64, 0, st>>>(res_partial, nblk, mq, res_out);
    return cudaGetLastError();
}

// ------------------------------------------------------- one-CTA m x m work
// Equilibrated Cholesky G~ = D G D = R~^H R~ (upper R~), R^-1 = D R~^-1;
// mode 1 adds the generalized Rayleigh-Ritz: Hhat = R^-H S R^-1, cyclic
// parallel (round-robin) complex Jacobi, Q = R^-1 Qhat, theta ascending.
__device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }

__global__ void __launch_bounds__(kThreads) small_kernel(const double2* __restrict__ G,
                                                        const double2* __restrict__ S, int m,
                                                        int mode, double2* __restrict__ Qout,
                                                        double* __restrict__ theta,
                                                        int* __restrict__ flags) {
    extern __shared__ double2 sm[];
    double2* A0 = sm;
    double2* A1 = sm + m * m;
    double2* A2 = sm + 2 * m * m;
    __shared__ double dsc[KHP_MAX_M];
    __shared__ int fail;
    __shared__ double red[kThreads];
    __shared__ int rp[KHP_MAX_M / 2], rq[KHP_MAX_M / 2];
    __shared__ double rc[KHP_MAX_M / 2], rs[KHP_MAX_M / 2];
    __shared__ double2 re[KHP_MAX_M / 2];
    __shared__ int perm[KHP_MAX_M];
    const int tid = threadIdx.x;
    const int mm = m * m;

    if (tid == 0) fail = 0;
    __syncthreads();
    if (tid < m) {
        const double d = G[tid * m + tid].x;
        if (!(d > 0.0) || !isfinite(d)) {
            dsc[tid] = 1.0;
            atomicOr(&fail, 1);
        } else {
            dsc[tid] = rsqrt(d);
        }
    }
    __syncthreads();
    if (fail) {
        if (tid == 0) atomicOr(flags, 2 | 4);
        return;
    }

    // ---- Cholesky (shift retried once on a non-positive pivot)
    for (int attempt = 0; attempt < 2; ++attempt) {
        const double shift = attempt == 0 ? 0.0 : 1e-11;
        for (int idx = tid; idx < mm; idx += kThreads) {
            const int i = idx / m, j = idx - i * m;
            double2 g = G[idx];
            g.x *= dsc[i] * dsc[j];
            g.y *= dsc[i] * dsc[j];
            if (i == j) { g.x += shift; g.y = 0.0; }
            A0[idx] = g;
        }
        if (tid == 0) fail = 0;
        __syncthreads();
        for (int k = 0; k < m; ++k) {
            if (tid == 0) {
                const double piv = A0[k * m + k].x;
                if (!(piv > 1e-13) || !isfinite(piv)) fail = 1;
                else A0[k * m + k] = make_double2(sqrt(piv), 0.0);
            }
            __syncthreads();
            if (fail) break;
            const double r = A0[k * m + k].x;
            for (int j = k + 1 + tid; j < m; j += kThreads) {
                A0[k * m + j].x /= r;
                A0[k * m + j].y /= r;
            }
            __syncthreads();
            const int t = m - k - 1;
            for (int idx = tid; idx < t * t; idx += kThreads) {
                const int i = k + 1 + idx / t, j = k + 1 + idx % t;
                if (j >= i) {
                    const double2 a = A0[k * m + i], b = A0[k * m + j];
                    double2 c = A0[i * m + j];
                    // c -= conj(a) * b
                    c.x -= a.x * b.x + a.y * b.y;
                    c.y -= a.x * b.y - a.y * b.x;
                    A0[i * m + j] = c;
                }
            }
            __syncthreads();
        }
        if (!fail) break;
        if (attempt == 0 && tid == 0) atomicOr(flags, 1);
        __syncthreads();
    }
    if (fail) {
        if (tid == 0) atomicOr(flags, 2);
        return;
    }

    // ---- R~^-1 (upper), one column per thread; then R^-1 = D R~^-1 in A1
    if (tid < m) {
        const int j = tid;
        for (int i = m - 1; i > j; --i) A1[i * m + j] = make_double2(0.0, 0.0);
        A1[j * m + j] = make_double2(1.0 / A0[j * m + j].x, 0.0);
        for (int i = j - 1; i >= 0; --i) {
            double2 s = make_double2(0.0, 0.0);
            for (int k = i + 1; k <= j; ++k) cfma(s, A0[i * m + k], A1[k * m + j]);
            const double inv = 1.0 / A0[i * m + i].x;
            A1[i * m + j] = make_double2(-s.x * inv, -s.y * inv);
        }
    }
    __syncthreads();
    for (int idx = tid; idx < mm; idx += kThreads) {
        const int i = idx / m;
        A1[idx].x *= dsc[i];
        A1[idx].y *= dsc[i];
    }
    __syncthreads();
    if (mode == 0) {
        for (int idx = tid; idx < mm; idx += kThreads) Qout[idx] = A1[idx];
        return;
    }

    // ---- Hhat = Rinv^H S Rinv
    for (int idx = tid; idx < mm; idx += kThreads) {        // A0 = S Rinv
        const int i = idx / m, j = idx - i * m;
        double2 s = make_double2(0.0, 0.0);
        for (int k = 0; k <= j; ++k) cfma(s, S[i * m + k], A1[k * m + j]);
        A0[idx] = s;
    }
    __syncthreads();
    for (int idx = tid; idx < mm; idx += kThreads) {        // A2 = Rinv^H A0
        const int i = idx / m, j = idx - i * m;
        double2 s = make_double2(0.0, 0.0);
        for (int k = 0; k <= i; ++k) cfmac(s, A1[k * m + i], A0[k * m + j]);
        A2[idx] = s;
    }
    __syncthreads();
    for (int idx = tid; idx < mm; idx += kThreads) {        // Hermitian part; V = I in A0
        const int i = idx / m, j = idx - i * m;
        if (j > i) {
            const double2 a = A2[i * m + j], b = A2[j * m + i];
            const double2 h = make_double2(0.5 * (a.x + b.x), 0.5 * (a.y - b.y));
            A2[i * m + j] = h;
            A2[j * m + i] = cconj(h);
        } else if (j == i) {
            A2[idx].y = 0.0;
        }
        A0[idx] = make_double2(i == j ? 1.0 : 0.0, 0.0);
    }
    __syncthreads();

    // ---- cyclic round-robin Jacobi
    const int me = (m + 1) & ~1;         // players (even); index m is a dummy when m is odd
    const int np = me / 2;
    for (int sweep = 0; sweep < 60; ++sweep) {
        double off = 0.0, dia = 0.0;
        for (int idx = tid; idx < mm; idx += kThreads) {
            const int i = idx / m, j = idx - i * m;
            const double2 a = A2[idx];
            if (i == j) dia += a.x * a.x;
            else off += a.x * a.x + a.y * a.y;
        }
        red[tid] = off;
        __syncthreads();
        for (int s = kThreads / 2; s > 0; s >>= 1) {
            if (tid < s) red[tid] += red[tid + s];
            __syncthreads();
        }
        const double offs = red[0];
        __syncthreads();
        red[tid] = dia;
        __syncthreads();
        for (int s = kThreads / 2; s > 0; s >>= 1) {
            if (tid < s) red[tid] += red[tid + s];
            __syncthreads();
        }
        const double dias = red[0];
        __syncthreads();
        if (offs <= 1e-32 * dias || offs == 0.0) break;

        for (int round = 0; round < me - 1; ++round) {
            if (tid < np) {
                int p, q;
                if (tid == 0) {
                    p = 0;
                    q = round % (me - 1) + 1;
                } else {
                    p = (round + tid) % (me - 1) + 1;
                    q = (round + me - 1 - tid) % (me - 1) + 1;
                }
                if (p > q) { const int t = p; p = q; q = t; }
                double c = 1.0, s = 0.0, t = 0.0;
                double2 e = make_double2(1.0, 0.0);
                if (q < m) {
                    const double a = A2[p * m + p].x, b = A2[q * m + q].x;
                    const double2 apq = A2[p * m + q];
                    const double g = hypot(apq.x, apq.y);
                    if (g > 0.0 && g > 1e-300) {
                        const double tau = (b - a) / (2.0 * g);
                        t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                        c = 1.0 / sqrt(1.0 + t * t);
                        s = t * c;
                        e = make_double2(apq.x / g, apq.y / g);
                    }
                }
                rp[tid] = p; rq[tid] = q; rc[tid] = c; rs[tid] = s; re[tid] = e;
            }
            __syncthreads();
            // columns: A <- A J, V <- V J ; J_pp=c, J_pq=s, J_qp=-s conj(e), J_qq=c conj(e)
            for (int idx = tid; idx < np * m; idx += kThreads) {
                const int k = idx / m, i = idx - k * m;
                const int p = rp[k], q = rq[k];
                if (q >= m || rs[k] == 0.0) continue;
                const double c = rc[k], s = rs[k];
                const double2 ec = cconj(re[k]);
                {
                    const double2 ap = A2[i * m + p], aq = A2[i * m + q];
                    const double2 aqe = cmul(aq, ec);
                    A2[i * m + p] = make_double2(c * ap.x - s * aqe.x, c * ap.y - s * aqe.y);
                    A2[i * m + q] = make_double2(s * ap.x + c * aqe.x, s * ap.y + c * aqe.y);
                }
                {
                    const double2 vp = A0[i * m + p], vq = A0[i * m + q];
                    const double2 vqe = cmul(vq, ec);
                    A0[i * m + p] = make_double2(c * vp.x - s * vqe.x, c * vp.y - s * vqe.y);
                    A0[i * m + q] = make_double2(s * vp.x + c * vqe.x, s * vp.y + c * vqe.y);
                }
            }
            __syncthreads();
            // rows: A <- J^H A ; (J^H)_pp=c, (J^H)_pq=-s e, (J^H)_qp=s, (J^H)_qq=c e
            for (int idx = tid; idx < np * m; idx += kThreads) {
                const int k = idx / m, j = idx - k * m;
                const int p = rp[k], q = rq[k];
                if (q >= m || rs[k] == 0.0) continue;
                const double c = rc[k], s = rs[k];
                const double2 e = re[k];
                const double2 ap = A2[p * m + j], aq = A2[q * m + j];
                const double2 aqe = cmul(e, aq);
                A2[p * m + j] = make_double2(c * ap.x - s * aqe.x, c * ap.y - s * aqe.y);
                A2[q * m + j] = make_double2(s * ap.x + c * aqe.x, s * ap.y + c * aqe.y);
            }
            __syncthreads();
            // exact 2x2 result on the pivots
            if (tid < np) {
                const int p = rp[tid], q = rq[tid];
                if (q < m && rs[tid] != 0.0) {
                    const double2 apq0 = A2[p * m + q];
                    (void)apq0;
                    A2[p * m + q] = make_double2(0.0, 0.0);
                    A2[q * m + p] = make_double2(0.0, 0.0);
                    A2[p * m + p].y = 0.0;
                    A2[q * m + q].y = 0.0;
                }
            }
            __syncthreads();
        }
    }

    // ---- sort ascending, Q = Rinv V(:, perm)
    if (tid == 0) {
        for (int i = 0; i < m; ++i) perm[i] = i;
        for (int i = 0; i < m; ++i) {
            int best = i;
            for (int k = i + 1; k < m; ++k)
                if (A2[perm[k] * m + perm[k]].x < A2[perm[best] * m + perm[best]].x) best = k;
            const int t = perm[i]; perm[i] = perm[best]; perm[best] = t;
        }
    }
    __syncthreads();
    if (tid < m) theta[tid] = A2[perm[tid] * m + perm[tid]].x;
    for (int idx = tid; idx < mm; idx += kThreads) {
        const int i = idx / m, k = idx - i * m;
        const int col = perm[k];
        double2 s = make_double2(0.0, 0.0);
        for (int l = i; l < m; ++l) cfma(s, A1[i * m + l], A0[l * m + col]);
        Qout[idx] = s;
    }
    bool finite = true;
    if (tid < m) finite = isfinite(A2[tid * m + tid].x);
    if (!finite) atomicOr(flags, 4);
}

cudaError_t launch_small(const double2* G, const double2* S, int m, int mode, double2* Q,
                         double* theta, int* flags, cudaStream_t st) {
    static bool attr_set = false;
    if (!attr_set) {
        cudaFuncSetAttribute(small_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        attr_set = true;
    }
    const size_t smem = 3ull * m * m * sizeof(double2);
    small_kernel<<<1, kThreads, smem, st>>>(G, S, m, mode, Q, theta, flags);
    return cudaGetLastError();
}

// ------------------------------------------------------------- utilities
// Precision conversion of columns [col0, col0 + ncol) of a row-major block.
__global__ void d2f_kernel(const double2* __restrict__ s, float2* __restrict__ d, long long rows, int ld,
                           int col0, int ncol) {
    const long long n = rows * ncol;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const long long r = i / ncol;
        const long long k = r * ld + col0 + (i - r * ncol);
        const double2 v = s[k];
        d[k] = make_float2((float)v.x, (float)v.y);
    }
}
__global__ void f2d_kernel(const float2* __restrict__ s, double2* __restrict__ d, long long rows, int ld,
                           int col0, int ncol) {
    const long long n = rows * ncol;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const long long r = i / ncol;
        const long long k = r * ld + col0 + (i - r * ncol);
        const float2 v = s[k];
        d[k] = make_double2((double)v.x, (double)v.y);
    }
}

static unsigned grid_for(long long n) {
    long long b = (n + 255) / 256;
    if (b > 148 * 16) b = 148 * 16;
    if (b < 1) b = 1;
    return (unsigned)b;
}

cudaError_t launch_convert_d2f(const double2* src, float2* dst, long long rows, int ld, int col0, int ncol,
                               cudaStream_t st) {
    d2f_kernel<<<grid_for(rows * ncol), 256, 0, st>>>(src, dst, rows, ld, col0, ncol);
    return cudaGetLastError();
}
cudaError_t launch_convert_f2d(const float2* src, double2* dst, long long rows, int ld, int col0, int ncol,
                               cudaStream_t st) {
    f2d_kernel<<<grid_for(rows * ncol), 256, 0, st>>>(src, dst, rows, ld, col0, ncol);
    return cudaGetLastError();
}

// SplitMix64 (Steele, Lea, Flood 2014): a counter-based 64-bit mixer.
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long z) {
    z += 0x9e3779b97f4a7c15ULL;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

__global__ void random_fill_kernel(double2* X, long long rows, int ld, int col0, int ncol,
                                   unsigned long long seed, const uint8_t* mask, int bands) {
    const long long n = rows * ncol;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const long long r = i / ncol;
        const int c = (int)(i - r * ncol);
        double2 v = make_double2(0.0, 0.0);
        if (!mask || mask[r / bands]) {
            const unsigned long long h = splitmix64(seed * 0x632be59bd9b4e019ULL + (unsigned long long)(r * 64 + col0 + c));
            const double u1 = (double)(h >> 11) * (1.0 / 9007199254740992.0);
            const unsigned long long h2 = splitmix64(h);
            const double u2 = (double)(h2 >> 11) * (1.0 / 9007199254740992.0);
            v = make_double2(2.0 * u1 - 1.0, 2.0 * u2 - 1.0);
        }
        X[r * ld + col0 + c] = v;
    }
}

cudaError_t launch_random_fill(double2* X, long long rows, int ld, int col0, int ncol,
                               unsigned long long seed, const uint8_t* mask, cudaStream_t st, int bands) {
    random_fill_kernel<<<grid_for(rows * ncol), 256, 0, st>>>(X, rows, ld, col0, ncol, seed, mask, bands);
    return cudaGetLastError();
}

}  // namespace khp

namespace khp {

// ------------------------------------------------------ Lanczos upper bound
// Three-term Lanczos on one vector, every scalar kept on the device:
//   w = H v_j ; alpha_j = Re v_j^H w ; w -= alpha_j v_j + beta_{j-1} v_{j-1} ;
//   beta_j = |w| ; v_{j+1} = w / beta_j
// The k x k tridiagonal matrix is then diagonalised by the one-CTA kernel.
__global__ void dot_re_partial(const double2* __restrict__ a, const double2* __restrict__ b, long long n,
                               double* __restrict__ partial) {
    __shared__ double red[256];
    const long long per = (n + gridDim.x - 1) / gridDim.x;
    const long long i0 = (long long)blockIdx.x * per;
    const long long i1 = i0 + per < n ? i0 + per : n;
    double s = 0.0;
    for (long long i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
        const double2 x = a[i], y = b[i];
        s += x.x * y.x + x.y * y.y;
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int k = 128; k > 0; k >>= 1) {
        if (threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

// out[0] = sum (mode 0) or sqrt(sum) (mode 1)
__global__ void finish_sum(const double* __restrict__ partial, int nb, double* out, int mode) {
    __shared__ double red[256];
    double s = 0.0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) s += partial[i];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int k = 128; k > 0; k >>= 1) {
        if (threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = mode == 1 ? sqrt(red[0]) : red[0];
}

// w -= alpha v + beta vprev (vprev may be null); partial |w|^2
__global__ void lanczos_update(double2* __restrict__ w, const double2* __restrict__ v,
                               const double2* __restrict__ vprev, const double* __restrict__ alpha,
                               const double* __restrict__ beta, long long n, double* __restrict__ partial) {
    __shared__ double red[256];
    const double al = *alpha, be = vprev ? *beta : 0.0;
    const long long per = (n + gridDim.x - 1) / gridDim.x;
    const long long i0 = (long long)blockIdx.x * per;
    const long long i1 = i0 + per < n ? i0 + per : n;
    double s = 0.0;
    for (long long i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
        double2 x = w[i];
        const double2 y = v[i];
        x.x -= al * y.x;
        x.y -= al * y.y;
        if (vprev) {
            const double2 z = vprev[i];
            x.x -= be * z.x;
            x.y -= be * z.y;
        }
        w[i] = x;
        s += x.x * x.x + x.y * x.y;
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int k = 128; k > 0; k >>= 1) {
        if (threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

__global__ void scale_vec(double2* __restrict__ dst, const double2* __restrict__ src,
                          const double* __restrict__ nrm, long long n) {
    const double inv = 1.0 / *nrm;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const double2 x = src[i];
        dst[i] = make_double2(x.x * inv, x.y * inv);
    }
}

// G = I, S = tridiag(beta, alpha, beta) as complex k x k matrices
__global__ void build_tridiag(const double* __restrict__ alpha, const double* __restrict__ beta, int k,
                              double2* __restrict__ G, double2* __restrict__ S) {
    for (int idx = threadIdx.x; idx < k * k; idx += blockDim.x) {
        const int i = idx / k, j = idx - i * k;
        G[idx] = make_double2(i == j ? 1.0 : 0.0, 0.0);
        double v = 0.0;
        if (i == j) v = alpha[i];
        else if (j == i + 1) v = beta[i];
        else if (i == j + 1) v = beta[j];
        S[idx] = make_double2(v, 0.0);
    }
}

static constexpr int kLzBlocks = 296;

cudaError_t lanczos_dot(const double2* a, const double2* b, long long n, double* partial, double* out,
                        cudaStream_t st) {
    dot_re_partial<<<kLzBlocks, 256, 0, st>>>(a, b, n, partial);
    finish_sum<<<1, 256, 0, st>>>(partial, kLzBlocks, out, 0);
    return cudaGetLastError();
}

cudaError_t lanczos_orth(double2* w, const double2* v, const double2* vprev, const double* alpha,
                         const double* beta_prev, double* beta_out, long long n, double* partial,
                         cudaStream_t st) {
    lanczos_update<<<kLzBlocks, 256, 0, st>>>(w, v, vprev, alpha, beta_prev, n, partial);
    finish_sum<<<1, 256, 0, st>>>(partial, kLzBlocks, beta_out, 1);
    return cudaGetLastError();
}

cudaError_t lanczos_norm(const double2* v, long long n, double* partial, double* out, cudaStream_t st) {
    dot_re_partial<<<kLzBlocks, 256, 0, st>>>(v, v, n, partial);
    finish_sum<<<1, 256, 0, st>>>(partial, kLzBlocks, out, 1);
    return cudaGetLastError();
}

cudaError_t lanczos_scale(double2* dst, const double2* src, const double* nrm, long long n, cudaStream_t st) {
    scale_vec<<<grid_for(n), 256, 0, st>>>(dst, src, nrm, n);
    return cudaGetLastError();
}

cudaError_t lanczos_tridiag(const double* alpha, const double* beta, int k, double2* G, double2* S,
                            cudaStream_t st) {
    build_tridiag<<<1, 256, 0, st>>>(alpha, beta, k, G, S);
    return cudaGetLastError();
}

}  // namespace khp

namespace khp {

// ------------------------------------------- defect-corrected FP32 filter
// For Ritz pairs (theta_c, x_c) with residual r_c = H x_c - theta_c x_c, the
// filtered block is Y_k = X diag(D_k) + Z_k, D_k the scalar recurrence at the
// Ritz values and Z_{k+1} = alpha_k (H - c) Z_k + gamma_k Z_{k-1} + alpha_k R D_k.
// These kernels form R (and Z_1 = alpha_0 R) in FP32 from the FP64 pair, and
// recombine Y = X D + Z in FP64 (W = H Y then comes from one FP64 apply:
// forming H Z in FP32 would cap the accuracy near 1e-9 eV).
struct DcResidualArgs {
    const double2* X;
    const double2* HX;
    float2* R;
    float2* Z1;
    long long rows;
    int ld, col0, ncol;
    double theta[64];
    double alpha0;
};

__global__ void dc_residual_kernel(const DcResidualArgs a) {
    const long long n = a.rows * a.ncol;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const long long r = i / a.ncol;
        const int c = a.col0 + (int)(i - r * a.ncol);
        const long long k = r * a.ld + c;
        const double2 x = a.X[k], hx = a.HX[k];
        const double th = a.theta[c];
        const double rx = hx.x - th * x.x, ry = hx.y - th * x.y;
        a.R[k] = make_float2((float)rx, (float)ry);
        a.Z1[k] = make_float2((float)(a.alpha0 * rx), (float)(a.alpha0 * ry));
    }
}

struct DcCombineArgs {
    const double2* X;
    const double2* HX;
    const float2* Z;
    double2* Y;
    double2* W;
    long long rows;
    int ld, zcol0;   // columns >= zcol0 carry Z; W is written for columns < zcol0 only
    double D[64];
};

__global__ void dc_combine_kernel(const DcCombineArgs a) {
    const long long n = a.rows * a.ld;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(i % a.ld);
        const double2 x = a.X[i];
        if (c >= a.zcol0) {
            const double d = a.D[c];
            const float2 z = a.Z[i];
            a.Y[i] = make_double2(fma(d, x.x, (double)z.x), fma(d, x.y, (double)z.y));
        } else {
            a.Y[i] = x;          // locked column: unchanged, with its H x
            a.W[i] = a.HX[i];
        }
    }
}

cudaError_t launch_dc_residual(const double2* X, const double2* HX, float2* R, float2* Z1, long long rows,
                               int ld, int col0, int ncol, const double* theta, double alpha0,
                               cudaStream_t st) {
    DcResidualArgs a;
    a.X = X; a.HX = HX; a.R = R; a.Z1 = Z1; a.rows = rows; a.ld = ld; a.col0 = col0; a.ncol = ncol;
    for (int c = 0; c < 64; ++c) a.theta[c] = c < ld ? theta[c] : 0.0;
    a.alpha0 = alpha0;
    dc_residual_kernel<<<grid_for(rows * ncol), 256, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_dc_combine(const double2* X, const double2* HX, const float2* Z, double2* Y, double2* W,
                              long long rows, int ld, int zcol0, const double* D, cudaStream_t st) {
    DcCombineArgs a;
    a.X = X; a.HX = HX; a.Z = Z; a.Y = Y; a.W = W; a.rows = rows; a.ld = ld; a.zcol0 = zcol0;
    for (int c = 0; c < 64; ++c) a.D[c] = c < ld ? D[c] : 0.0;
    dc_combine_kernel<<<grid_for(rows * ld), 256, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace khp
