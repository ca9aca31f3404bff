"""Rayleigh-Ritz contractions on the tensor cores (split-digit BF16 products
recombined in FP64) against FP64 references: the Gram matrices G = Y^H Y,
S = Y^H (H Y) and the rotation X = Y Q, through the C-ABI (khp_project,
khp_rotate), and the eigensolver with each projection path.  Method 0 is
the tcgen05 path (accumulators in TMEM), 2 the mma.sync path, 1 FP64 ALU.

Accuracy bar: the split keeps 49 bits below each block's exponent bound and
accumulates exactly, so each entry must agree with an extended-precision
reference to a few units of 2^-49 of the norm scale of that entry; FP64
BLAS on the same data is held to the same bar.
"""
import numpy as np
import pytest
import torch

import inputs
from oracle import kp

pytestmark = pytest.mark.gpu

GRID = (37, 19, 14)      # 59,052 rows: many 64-row chunks and a ragged tail
EPS49 = 2.0 ** -49


def _grid(khp):
    p = inputs.small_problem(*GRID, h=0.5, seed=21, rot="device", B=(0.3, 0.0, 0.4), gauge=0, strain=True)
    return p, khp.KPGrid.from_problem(p)


def _block(n, m, seed, col_scale=None, row_scale=None):
    Y = inputs.random_block(n, m, seed=seed)
    if col_scale is not None:
        Y = Y * col_scale[None, :]
    if row_scale is not None:
        Y = Y * row_scale[:, None]
    return Y


def _gram_ref(Y, W):
    """Y^H W in extended precision (numpy longdouble accumulation)."""
    Yl = Y.real.astype(np.longdouble), Y.imag.astype(np.longdouble)
    Wl = W.real.astype(np.longdouble), W.imag.astype(np.longdouble)
    re = Yl[0].T @ Wl[0] + Yl[1].T @ Wl[1]
    im = Yl[0].T @ Wl[1] - Yl[1].T @ Wl[0]
    return re, im


def _herm_upper(re, im):
    """The Hermitian matrix built from the upper triangle (as the library does)."""
    m = re.shape[0]
    out = np.zeros((m, m), dtype=np.complex128)
    for i in range(m):
        for j in range(i, m):
            out[i, j] = complex(float(re[i, j]), float(im[i, j]))
            out[j, i] = np.conj(out[i, j]) if i != j else complex(float(re[i, i]), 0.0)
    return out


def _check_gram(G, Y, W):
    re, im = _gram_ref(Y, W)
    ref = _herm_upper(re, im)
    ny = np.linalg.norm(Y, axis=0)
    nw = np.linalg.norm(W, axis=0)
    scale = np.maximum(np.outer(ny, nw), np.outer(nw, ny))
    err = np.abs(G - ref) / np.where(scale > 0, scale, 1.0)
    return err.max()


@pytest.mark.parametrize("method", [0, 2])
def test_gram_worst_case_digit_patterns(khp, method):
    """The exact FP32 accumulation of the digit products holds at its bound:
    every entry of Y equal to the largest value whose 49-bit balanced
    base-128 digits are all extreme and of one sign (leading digit 127, the
    others +63), so that every digit product of a level has the same sign
    and every row sits at its exponent block's maximum.  G = Y^H Y is then
    N v^2 (up to the sign pattern of the columns), computed exactly in
    integers here."""
    p, g = _grid(khp)
    N, m = p.n_unknowns, 24
    # F = 2^49 - 1 - (64 + 64*128 + ... + 64*128^5): digits u_s = 127 of
    # F + the balancing offset; v = 16 F / 2^52 lies in [1, 2)
    bal = sum(64 * 128 ** k for k in range(6))
    F = 2 ** 49 - 1 - bal
    mant = 16 * F
    v = mant / 2.0 ** 52
    assert 1.0 <= v < 2.0 and float(mant) == mant
    signs = np.where(np.arange(m) % 3 == 1, -1.0, 1.0)
    Y = np.empty((N, m), dtype=np.complex128)
    Y.real = v * signs[None, :]
    Y.imag = v * signs[None, ::-1]
    G, _ = g.project(Y, None, method=method)
    # exact: G_ij = N v^2 (s_i s_j + t_i t_j) + i N v^2 (s_i t_j - t_i s_j)
    t = signs[::-1]
    v2 = mant * mant                                  # v^2 = v2 / 2^104, exact integer
    for i in range(m):
        for j in range(m):
            re = N * v2 * int(signs[i] * signs[j] + t[i] * t[j])
            im = N * v2 * int(signs[i] * t[j] - t[i] * signs[j])
            ref = complex(re / 2.0 ** 104, im / 2.0 ** 104)
            scale = 2 * N * v * v
            assert abs(G[i, j] - ref) <= 4 * EPS49 * scale, (i, j, G[i, j], ref)


@pytest.mark.parametrize("m", [1, 5, 8, 12, 24, 32])
def test_gram_matches_extended_precision(khp, m):
    p, g = _grid(khp)
    Y = _block(p.n_unknowns, m, seed=40 + m)
    W = g.apply(torch.from_numpy(Y)).cpu().numpy()
    for method in (0, 1, 2):
        G, S = g.project(Y, W, method=method)
        assert _check_gram(G, Y, Y) <= 16 * EPS49, method
        assert _check_gram(S, Y, W) <= 16 * EPS49, method
        # without W the kernel may pick longer exponent blocks: same accuracy bar
        Gonly, none = g.project(Y, None, method=method)
        assert none is None
        assert _check_gram(Gonly, Y, Y) <= 16 * EPS49, method


@pytest.mark.parametrize("method", [0, 2])
def test_gram_column_scales_and_zero_columns(khp, method):
    """Columns spread over 60 decades, one all-zero column: the per-chunk
    column exponents keep every entry accurate relative to its own norms."""
    p, g = _grid(khp)
    m = 24
    cs = 10.0 ** np.linspace(-30, 30, m)
    cs[7] = 0.0
    Y = _block(p.n_unknowns, m, seed=77, col_scale=cs)
    W = g.apply(torch.from_numpy(Y)).cpu().numpy()
    G, S = g.project(Y, W, method=method)
    assert _check_gram(G, Y, Y) <= 16 * EPS49
    assert _check_gram(S, Y, W) <= 16 * EPS49
    assert np.all(G[7] == 0) and np.all(G[:, 7] == 0)


@pytest.mark.parametrize("method", [0, 2])
def test_gram_propagates_nan(khp, method):
    p, g = _grid(khp)
    Y = _block(p.n_unknowns, 8, seed=5)
    Y[1234, 3] = np.nan
    G, _ = g.project(Y, None, method=method)
    assert np.isnan(G[3, 3].real)
    assert np.isfinite(G[0, 1]) and np.isfinite(G[5, 6])


@pytest.mark.parametrize("m", [1, 5, 12, 24, 32])
def test_rotation_matches_extended_precision(khp, m):
    p, g = _grid(khp)
    rs = 10.0 ** np.random.default_rng(3).uniform(-20, 20, p.n_unknowns)
    Y = _block(p.n_unknowns, m, seed=60 + m, row_scale=rs)
    W = _block(p.n_unknowns, m, seed=160 + m)
    rng = np.random.default_rng(m)
    Q = rng.standard_normal((m, m)) + 1j * rng.standard_normal((m, m))
    Q[:, 0] *= 1e-12
    Ql = Q.real.astype(np.longdouble), Q.imag.astype(np.longdouble)
    for method in (0, 1, 2):
        X, HX = g.rotate(Y, Q, W, method=method)
        for A, B in ((Y, X), (W, HX)):
            Al = A.real.astype(np.longdouble), A.imag.astype(np.longdouble)
            ref_re = Al[0] @ Ql[0] - Al[1] @ Ql[1]
            ref_im = Al[0] @ Ql[1] + Al[1] @ Ql[0]
            B = B.cpu().numpy()
            scale = np.outer(np.linalg.norm(A, axis=1), np.linalg.norm(Q, axis=0))
            scale = np.where(scale > 0, scale, 1.0)
            err = np.maximum(np.abs(B.real - ref_re.astype(np.float64)), np.abs(B.imag - ref_im.astype(np.float64)))
            assert (err / scale).max() <= 16 * EPS49, method


@pytest.mark.parametrize("method", [0, 2])
def test_rotation_in_place(khp, method):
    p, g = _grid(khp)
    m = 24
    Y = torch.from_numpy(_block(p.n_unknowns, m, seed=9)).cuda()
    W = torch.from_numpy(_block(p.n_unknowns, m, seed=10)).cuda()
    rng = np.random.default_rng(1)
    Q = rng.standard_normal((m, m)) + 1j * rng.standard_normal((m, m))
    X_ref, HX_ref = g.rotate(Y, Q, W, method=method)
    g.rotate(Y, Q, W, method=method, out=Y, out_w=W)
    assert torch.equal(Y, X_ref) and torch.equal(W, HX_ref)


def test_rotation_without_w_and_nan(khp):
    """X = Y Q alone (the re-orthonormalisation), and a NaN in one row of Y
    reaching only that row of X."""
    p, g = _grid(khp)
    m = 16
    Y = _block(p.n_unknowns, m, seed=12)
    Y[777, 2] = np.nan
    rng = np.random.default_rng(4)
    Q = rng.standard_normal((m, m)) + 1j * rng.standard_normal((m, m))
    X, HX = g.rotate(Y, Q, None, method=0)
    assert HX is None
    X = X.cpu().numpy()
    assert np.isnan(X[777]).all()
    ok = np.ones(p.n_unknowns, dtype=bool)
    ok[777] = False
    ref = Y[ok] @ Q
    scale = np.outer(np.linalg.norm(Y[ok], axis=1), np.linalg.norm(Q, axis=0))
    assert (np.abs(X[ok] - ref) / scale).max() <= 16 * EPS49


@pytest.mark.parametrize("case", ["config1", "field"])
def test_eigensolve_tensor_vs_fp64_projections(khp, case):
    if case == "config1":
        p = inputs.config1()
        kw = dict(n_states=p.n_states, block_m=p.block_m, degree=p.degree)
    else:
        p = inputs.small_problem(12, 9, 8, h=0.5, seed=4, rot="device", B=(0.5, 0.2, 0.0), gauge=0, strain=True)
        kw = dict(n_states=8, block_m=16, degree=16)
    g = khp.KPGrid.from_problem(p)
    rt = g.eigensolve(**kw, tol=1e-10, seed=2, projections="tensor")
    rf = g.eigensolve(**kw, tol=1e-10, seed=2, projections="fp64")
    rm = g.eigensolve(**kw, tol=1e-10, seed=2, projections="mma")
    assert rt.stats["converged"] == kw["n_states"]
    assert np.abs(rt.evals - rf.evals).max() <= 1e-12
    assert np.abs(rm.evals - rf.evals).max() <= 1e-12
    H = kp.assemble(p)
    V = rt.evecs.cpu().numpy()
    res = np.linalg.norm(H @ V - V * rt.evals[None, :], axis=0)
    assert res.max() <= 1e-9
    assert np.abs(V.conj().T @ V - np.eye(V.shape[1])).max() < 1e-12


def test_project_rejects_bad_arguments(khp):
    p, g = _grid(khp)
    Y = _block(p.n_unknowns, 40, seed=1)
    with pytest.raises(khp.KHPError):
        g.project(Y, None, method=0)         # tensor-core path takes m <= 32
    with pytest.raises(khp.KHPError):
        g.project(Y[:, :8], None, method=3)
