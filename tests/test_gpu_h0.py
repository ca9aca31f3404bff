"""Spin-independent H0 (Sec. II C, Eq. 6a; three bands per point, no
spin-orbit, B = 0) through the CUDA path, against the FP64 oracle
(`kp.assemble_h0`): the stencil in FP64 and FP32, the eigensolver (plain and
defect-corrected FP32 filter), the density and the Hellmann-Feynman
gradients.  Sizes span several thread blocks with ragged tails."""
import numpy as np
import pytest
import torch

import inputs
from oracle import eig, kp, observables
from tests.metrics import clusters, subspace_sin_angle

pytestmark = pytest.mark.gpu

CASES = [
    dict(shape=(13, 7, 5), rot="identity", strain=True, mask=False),
    dict(shape=(9, 11, 6), rot="device", strain=True, mask=False),
    dict(shape=(10, 5, 7), rot="identity", strain=False, mask=True),
]


def _problem(c, seed=5, levers=0):
    return inputs.small_problem(*c["shape"], h=0.5, seed=seed, rot=c["rot"], strain=c["strain"],
                                mask=c["mask"], levers=levers)


def _grid(khp, p):
    return khp.KPGrid.from_problem(p, bands=3)


@pytest.mark.parametrize("case", range(len(CASES)))
@pytest.mark.parametrize("m", [1, 6, 24])
def test_h0_stencil_fp64_matches_csr(khp, case, m):
    p = _problem(CASES[case])
    H = kp.assemble_h0(p)
    X = inputs.random_block(3 * p.n_points, m, seed=400 + m)
    if p.mask is not None:
        X[np.repeat(p.mask.reshape(-1) == 0, 3)] = 0.0
    ref = H @ X
    g = _grid(khp, p)
    assert g.N == 3 * p.n_points
    Y = g.apply(torch.from_numpy(X), precision=0).cpu().numpy()
    assert np.abs(Y - ref).max() <= 1e-13 * np.abs(ref).max()


@pytest.mark.parametrize("case", range(len(CASES)))
@pytest.mark.parametrize("m", [2, 7, 24])
def test_h0_stencil_fp32_matches_csr(khp, case, m):
    p = _problem(CASES[case])
    H = kp.assemble_h0(p)
    X = inputs.random_block(3 * p.n_points, m, seed=500 + m).astype(np.complex64)
    if p.mask is not None:
        X[np.repeat(p.mask.reshape(-1) == 0, 3)] = 0.0
    ref = H @ X.astype(np.complex128)
    g = _grid(khp, p)
    Y = g.apply(torch.from_numpy(X), precision=1).cpu().numpy().astype(np.complex128)
    assert np.abs(Y - ref).max() <= 2e-5 * np.abs(ref).max()


@pytest.mark.parametrize("case", range(len(CASES)))
@pytest.mark.parametrize("precision", [0, 2])
def test_h0_eigensolve_matches_dense_oracle(khp, case, precision):
    p = _problem(CASES[case], seed=9)
    H = kp.assemble_h0(p)
    n = 8
    w, v = eig.lowest_dense(H, n + 2, mask=p.mask)
    g = _grid(khp, p)
    r = g.eigensolve(n, block_m=16, degree=16 if precision == 0 else 40, precision=precision, tol=1e-10, seed=4)
    assert r.stats["converged"] == n
    assert np.abs(r.evals - w[:n]).max() <= 1e-10
    V = r.evecs.cpu().numpy()
    assert np.abs(V.conj().T @ V - np.eye(n)).max() < 1e-12
    res = np.linalg.norm(H @ V - V * r.evals[None, :], axis=0)
    assert res.max() <= 1e-9
    for cl in clusters(w[:n]):
        if cl[-1] + 1 < len(w) and w[cl[-1] + 1] - w[cl[-1]] < 1e-6:
            continue
        assert subspace_sin_angle(v[:, cl], V[:, cl]) <= 1e-7


def test_h0_density_and_backward(khp):
    p = _problem(CASES[1], seed=3, levers=2)
    g = _grid(khp, p)
    n = 6
    r = g.eigensolve(n, block_m=16, degree=16, tol=1e-11, seed=2)
    V = r.evecs.cpu().numpy()
    wts = np.linspace(1.0, 0.5, n)
    rho = g.density(r.evecs, wts).cpu().numpy()
    assert np.abs(rho - observables.density(V, wts, bands=3)).max() <= 1e-14 * np.abs(rho).max()
    gw = np.ones(n)
    gw[0] -= 1.0
    gw[1] += 1.0
    lev = torch.from_numpy(p.levers.reshape(2, -1)).cuda()
    dV, dS, dA = g.backward(r.evecs, r.evals, gw, levers=lev)
    oV, oS, oA = observables.hf_gradients(V, gw, p.material, p.rot, p.levers, bands=3)
    assert np.abs(dV.cpu().numpy() - oV).max() <= 1e-12 * np.abs(oV).max()
    assert np.abs(dS.cpu().numpy().reshape(6, -1) - oS).max() <= 1e-12 * np.abs(oS).max()
    assert np.abs(dA - oA).max() <= 1e-12 * np.abs(oA).max()


def test_h0_rejects_magnetic_field(khp):
    p = _problem(CASES[0])
    g = _grid(khp, p)
    with pytest.raises(khp.KHPError):
        g.set_fields(p.V, p.strain, None, None, (0.0, 0.0, 0.1), 0)
