"""CUDA path vs the FP64 oracle, element by element, on seeded inputs.

Sizes are small enough for the dense oracle but span several thread blocks
and ragged tails in every direction; the cases cover both frames, both
gauges, B = 0 and B != 0, strain, a point mask, odd and even block widths,
and FP64 and FP32 stencils.
"""
import numpy as np
import pytest
import torch

import inputs
from oracle import eig, kp, observables
from tests.metrics import clusters, subspace_sin_angle

pytestmark = pytest.mark.gpu

CASES = [
    dict(shape=(13, 7, 5), rot="identity", B=(0, 0, 0), gauge=0, strain=True, mask=False),
    dict(shape=(9, 11, 6), rot="device", B=(0.5, 0.0, 0.0), gauge=0, strain=True, mask=False),
    dict(shape=(7, 6, 9), rot="device", B=(0.3, -0.8, 1.1), gauge=1, strain=True, mask=False),
    dict(shape=(10, 5, 7), rot="identity", B=(0.0, 0.7, 0.2), gauge=0, strain=False, mask=True),
    dict(shape=(33, 3, 4), rot="device", B=(0, 0, 0), gauge=0, strain=True, mask=True),
]


def _problem(c, seed=5):
    return inputs.small_problem(*c["shape"], h=0.5, seed=seed, rot=c["rot"], B=c["B"], gauge=c["gauge"],
                                strain=c["strain"], mask=c["mask"])


def _grid(khp, p):
    return khp.KPGrid.from_problem(p)


@pytest.mark.parametrize("case", range(len(CASES)))
@pytest.mark.parametrize("m", [1, 5, 8, 16, 20, 24, 32])
def test_stencil_fp64_matches_csr(khp, case, m):
    p = _problem(CASES[case])
    H = kp.assemble(p)
    X = inputs.random_block(p.n_unknowns, m, seed=100 + m)
    if p.mask is not None:
        X[np.repeat(p.mask.reshape(-1) == 0, 6)] = 0.0
    ref = H @ X
    g = _grid(khp, p)
    Y = g.apply(torch.from_numpy(X), precision=0).cpu().numpy()
    scale = np.abs(ref).max()
    assert np.abs(Y - ref).max() <= 1e-13 * scale


@pytest.mark.parametrize("case", range(len(CASES)))
@pytest.mark.parametrize("m", [2, 7, 16, 20, 24, 32])
def test_stencil_fp32_matches_csr(khp, case, m):
    p = _problem(CASES[case])
    H = kp.assemble(p)
    X = inputs.random_block(p.n_unknowns, m, seed=200 + m).astype(np.complex64)
    if p.mask is not None:
        X[np.repeat(p.mask.reshape(-1) == 0, 6)] = 0.0
    ref = H @ X.astype(np.complex128)
    g = _grid(khp, p)
    Y = g.apply(torch.from_numpy(X), precision=1).cpu().numpy().astype(np.complex128)
    # FP32 coefficients and arithmetic: a few ulps of the largest row terms
    scale = np.abs(ref).max() + 1e-30
    assert np.abs(Y - ref).max() <= 2e-6 * scale * 10


STEP_CASES = [
    # several 16 x 8 tiles with ragged edges in x and y, B along [110]
    dict(shape=(37, 19, 11), rot="device", B=(0.5, 0.0, 0.0), gauge=0, strain=True, mask=False),
    # exactly one tile, B = 0
    dict(shape=(16, 8, 3), rot="identity", B=(0, 0, 0), gauge=0, strain=True, mask=False),
    # tall in z (several z-chunks per tile), tilted field
    dict(shape=(5, 3, 30), rot="device", B=(0.2, 0.1, 0.4), gauge=0, strain=True, mask=False),
    # Landau gauge and a point mask: the per-point kernel
    dict(shape=(9, 11, 6), rot="device", B=(0.3, -0.8, 1.1), gauge=1, strain=True, mask=False),
    dict(shape=(10, 5, 7), rot="identity", B=(0.0, 0.7, 0.2), gauge=0, strain=False, mask=True),
]


@pytest.mark.parametrize("case", range(len(STEP_CASES)))
@pytest.mark.parametrize("ld,col0,ncol", [(24, 0, 24), (24, 6, 18), (20, 2, 13), (8, 0, 8), (6, 1, 4), (2, 0, 2)])
def test_filter_step_fp32_matches_oracle(khp, case, ld, col0, ncol):
    """The fused FP32 Chebyshev step of the defect-corrected filter,
    y = alpha H x + beta x + gamma prev + c_col src on columns
    [col0, col0 + ncol), against the oracle's CSR product in FP64 on the
    same (FP32) inputs; the other columns of y stay untouched."""
    p = _problem(STEP_CASES[case], seed=11)
    H = kp.assemble(p)
    N = p.n_unknowns
    x, prev, src, y0 = (inputs.random_block(N, ld, seed=300 + k).astype(np.complex64) for k in range(4))
    if p.mask is not None:
        x[np.repeat(p.mask.reshape(-1) == 0, 6)] = 0.0
    coef = np.random.default_rng(ld + col0).uniform(-1.0, 1.0, ld)
    alpha, beta, gamma = 0.37, -0.81, -0.55
    g = _grid(khp, p)
    y = torch.from_numpy(y0.copy()).cuda()
    g.filter_step(x, y, alpha, beta, gamma, prev=prev, src=src, src_coef=coef, col0=col0, ncol=ncol)
    Y = y.cpu().numpy()
    xd = x.astype(np.complex128)
    ref = alpha * (H @ xd) + beta * xd + gamma * prev.astype(np.complex128) + src.astype(np.complex128) * coef
    if p.mask is not None:
        ref[np.repeat(p.mask.reshape(-1) == 0, 6)] = 0.0
    cs = slice(col0, col0 + ncol)
    scale = np.abs(alpha * (H @ xd)).max() + np.abs(xd).max() + np.abs(prev).max() + np.abs(src).max()
    assert np.abs(Y[:, cs] - ref[:, cs]).max() <= 2e-6 * scale
    out = np.ones(ld, dtype=bool)
    out[cs] = False
    assert np.array_equal(Y[:, out], y0[:, out])


@pytest.mark.parametrize("case", [0, 3])
def test_filter_step_fp64_matches_oracle(khp, case):
    p = _problem(STEP_CASES[case], seed=12)
    H = kp.assemble(p)
    N, ld = p.n_unknowns, 12
    x, prev = inputs.random_block(N, ld, seed=401), inputs.random_block(N, ld, seed=402)
    g = _grid(khp, p)
    y = torch.zeros((N, ld), dtype=torch.complex128, device="cuda")
    g.filter_step(x, y, 0.4, 0.3, -0.9, prev=prev, col0=2, ncol=8, precision=0)
    ref = 0.4 * (H @ x) + 0.3 * x - 0.9 * prev
    Y = y.cpu().numpy()
    assert np.abs(Y[:, 2:10] - ref[:, 2:10]).max() <= 1e-13 * np.abs(ref).max()
    assert np.all(Y[:, :2] == 0) and np.all(Y[:, 10:] == 0)


def test_hermitian_matrix_free(khp):
    p = _problem(CASES[2])
    g = _grid(khp, p)
    x = torch.from_numpy(inputs.random_block(p.n_unknowns, 1, seed=1))
    y = torch.from_numpy(inputs.random_block(p.n_unknowns, 1, seed=2))
    Hx = g.apply(x).cpu()
    Hy = g.apply(y).cpu()
    a = (x.conj() * Hy).sum()
    b = (y.conj() * Hx).sum().conj()
    assert abs(a - b) <= 1e-13 * float(Hx.abs().max()) * x.numel() ** 0.5


def _check_solution(p, r, n, tol_e, tol_angle, oracle_w=None, oracle_v=None):
    H = kp.assemble(p)
    if oracle_w is None:
        oracle_w, oracle_v = eig.lowest_dense(H, n + 2, mask=p.mask)
    assert np.abs(r.evals - oracle_w[:n]).max() <= tol_e
    V = r.evecs.cpu().numpy()
    # orthonormal
    assert np.abs(V.conj().T @ V - np.eye(n)).max() < 1e-12
    # residuals through the oracle's CSR
    res = np.linalg.norm(H @ V - V * r.evals[None, :], axis=0)
    assert res.max() <= max(10 * r.stats["max_residual"], 1e-9)
    # invariant subspaces of whole clusters
    for cl in clusters(oracle_w[:n]):
        if cl[-1] + 1 < len(oracle_w) and oracle_w[cl[-1] + 1] - oracle_w[cl[-1]] < 1e-6:
            continue       # cluster cut at n: only its span is not unique
        assert subspace_sin_angle(oracle_v[:, cl], V[:, cl]) <= tol_angle
    return V


def test_eigensolve_config1_plain_fp64(khp):
    p = inputs.config1()
    g = _grid(khp, p)
    r = g.eigensolve(p.n_states, block_m=p.block_m, degree=p.degree, tol=1e-10, seed=3)
    _check_solution(p, r, p.n_states, 1e-10, 1e-7)
    assert r.stats["converged"] == p.n_states


@pytest.mark.parametrize("case", [1, 2, 3])
def test_eigensolve_field_strain_mask(khp, case):
    p = _problem(CASES[case], seed=9)
    g = _grid(khp, p)
    r = g.eigensolve(8, block_m=16, degree=16, tol=1e-10, seed=4)
    _check_solution(p, r, 8, 1e-10, 1e-7)


def test_eigensolve_config3_mixed(khp):
    p = inputs.config3()
    g = _grid(khp, p)
    r = g.eigensolve(p.n_states, block_m=p.block_m, degree=p.degree, precision=1,
                     refine_sweeps=p.refine_sweeps, tol=1e-10, seed=5)
    w, v = eig.lowest_dense(kp.assemble(p), p.n_states + 2)
    err = np.abs(r.evals - w[:p.n_states])
    assert err.max() <= 1e-7, err
    assert r.stats["iterations_fp32"] >= 1


def test_eigensolve_mixed_to_plain_tolerance(khp):
    p = inputs.config1()
    g = _grid(khp, p)
    r = g.eigensolve(p.n_states, block_m=16, degree=20, precision=1, refine_sweeps=-1, tol=1e-10, seed=6)
    _check_solution(p, r, p.n_states, 1e-10, 1e-7)


def test_warm_start_converges_immediately(khp):
    p = inputs.config1()
    g = _grid(khp, p)
    r0 = g.eigensolve(8, block_m=16, tol=1e-10, seed=7)
    r1 = g.eigensolve(8, block_m=16, tol=1e-10, seed=8, warm_start=r0.evecs)
    assert r1.stats["iterations"] <= 2
    assert np.abs(r1.evals - r0.evals).max() < 1e-11


def test_density_matches_oracle_same_vectors(khp):
    p = _problem(CASES[1])
    g = _grid(khp, p)
    V = inputs.random_block(p.n_unknowns, 6, seed=11)
    w = np.array([1.0, 0.5, -2.0, 0.25, 3.0, 1e-3])
    rho = g.density(torch.from_numpy(V), w).cpu().numpy()
    ref = observables.density(V, w)
    assert rho.shape == (p.n_points,)
    assert np.abs(rho - ref).max() <= 1e-12 * np.abs(ref).max()


def test_backward_matches_oracle_same_vectors(khp):
    p = inputs.small_problem(9, 7, 6, h=0.5, seed=3, rot="device", strain=True, levers=3)
    g = _grid(khp, p)
    V = inputs.random_block(p.n_unknowns, 4, seed=12)
    ev = np.array([0.0, 1.0, 2.0, 3.0])
    gr = np.array([1.5, -0.5, 2.0, 0.25])
    dV, dE, dA = g.backward(torch.from_numpy(V), ev, gr, levers=p.levers)
    rV, rE, rA = observables.hf_gradients(V, gr, p.material, p.rot, p.levers)
    assert np.abs(dV.cpu().numpy() - rV).max() <= 1e-12 * np.abs(rV).max()
    assert np.abs(dE.cpu().numpy().reshape(6, -1) - rE).max() <= 1e-12 * np.abs(rE).max()
    assert np.abs(dA - rA).max() <= 1e-12 * np.abs(rA).max()


def test_backward_rejects_split_cluster(khp):
    p = inputs.config1()
    g = _grid(khp, p)
    r = g.eigensolve(4, block_m=12, tol=1e-10)
    with pytest.raises(khp.KHPError) as ei:
        g.backward(r.evecs, r.evals, [1.0, 0.0, 0.0, 0.0])
    assert ei.value.status == 7


def test_autograd_gradient_vs_finite_difference(khp):
    """KPEigs backward (HF adjoint) vs central differences of the GPU solve,
    loss = doublet gap + sum of the lowest 8 (B = 0, doublet averages)."""
    p = inputs.small_problem(10, 8, 7, h=0.6, seed=4, rot="identity", strain=True, levers=3)
    g = khp.KPGrid(p.nx, p.ny, p.nz, p.h, p.material, p.rot)
    dev = torch.device("cuda")
    V = torch.tensor(p.V.reshape(-1), device=dev, requires_grad=True)
    S = torch.tensor(p.strain.reshape(6, -1), device=dev, requires_grad=True)
    A = torch.zeros(3, dtype=torch.float64, requires_grad=True)
    kw = dict(n_states=8, block_m=16, degree=16, tol=1e-11, seed=2)
    wts = torch.ones(8, dtype=torch.float64, device=dev)
    wts[0:2] -= 0.5
    wts[2:4] += 0.5

    def loss_of(Vv, Sv, Av):
        E = khp.KPEigs.apply(Vv, Sv, Av, g, p.levers, p.B, kw)
        return (E * wts).sum()

    L = loss_of(V, S, A)
    L.backward()
    rng = np.random.default_rng(0)
    d = 1e-5
    for _ in range(3):
        u = torch.tensor(rng.standard_normal(p.n_points), device=dev)
        fd = (loss_of(V.detach() + d * u, S.detach(), A.detach()) - loss_of(V.detach() - d * u, S.detach(), A.detach())) / (2 * d)
        an = (V.grad * u).sum()
        assert abs(float(fd - an)) <= 1e-6 * max(1.0, abs(float(fd)))
    for k in range(3):
        e = torch.zeros(3, dtype=torch.float64)
        e[k] = 1.0
        fd = (loss_of(V.detach(), S.detach(), A.detach() + d * e) - loss_of(V.detach(), S.detach(), A.detach() - d * e)) / (2 * d)
        assert abs(float(fd) - float(A.grad[k])) <= 1e-6 * max(1.0, abs(float(fd)))


def test_error_paths(khp):
    p = inputs.config1()
    g = khp.KPGrid(p.nx, p.ny, p.nz, p.h, p.material, p.rot)
    with pytest.raises(khp.KHPError) as ei:
        g.eigensolve(4, block_m=12)
    assert ei.value.status == 6                      # fields not set
    Vbad = p.V.copy()
    Vbad[0, 0, 0] = np.nan
    with pytest.raises(khp.KHPError) as ei:
        g.set_fields(Vbad)
    assert ei.value.status == 1
    g.set_fields(p.V)
    with pytest.raises(khp.KHPError) as ei:
        g.eigensolve(12, block_m=12)
    assert ei.value.status == 1                      # n >= m
    r = g.eigensolve(8, block_m=16, max_iter=2, tol=1e-12, allow_not_converged=True)
    assert r.status == 4 and r.stats["iterations"] == 2
    # the handle stays usable after every error
    r = g.eigensolve(8, block_m=16, tol=1e-10)
    assert r.status == 0


@pytest.mark.parametrize("case", [0, 2])
def test_spectral_upper_bound_is_an_upper_bound(khp, case):
    """The filter's upper bound (Lanczos, capped by Gershgorin) lies above
    the largest eigenvalue of the oracle's matrix, and not absurdly far."""
    p = _problem(CASES[case])
    wmax = eig.all_eigenvalues_dense(kp.assemble(p), mask=p.mask)[-1]
    g = _grid(khp, p)
    r = g.eigensolve(4, block_m=8, degree=8, tol=1e-6, max_iter=3, allow_not_converged=True)
    ub = r.stats["lambda_upper"]
    assert ub >= wmax
    assert ub <= 1.6 * wmax


@pytest.mark.parametrize("which", ["c1", 1, 2, 3])
def test_eigensolve_defect_corrected_fp32(khp, which):
    """precision 2: every filter apply in FP32 (defect-corrected by the FP64
    residual), FP64 projections; must reach the plain FP64 accuracy."""
    p = inputs.config1() if which == "c1" else _problem(CASES[which], seed=9)
    g = _grid(khp, p)
    r = g.eigensolve(8, block_m=16, degree=20, precision=2, tol=1e-10, seed=4)
    assert r.stats["launches_fp64"] == 0 and r.stats["launches_fp32"] > 0
    _check_solution(p, r, 8, 1e-10, 1e-7)
