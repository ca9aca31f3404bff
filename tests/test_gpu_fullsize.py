"""Full-size checks on the 160x48x48 workload (2.21M unknowns) in the launch
configuration bench.py times (16 states, block 24, degree 120, tol 1e-10 eV).

* eigenvalues against the stored FP64 oracle values (ARPACK, written by
  tests/golden/make_golden.py, which calls only the oracle);
* on the central 64x24x24 cut of the same fields: eigenvalues against the
  stored oracle values and the subspace angle against oracle eigenvectors;
* residuals recomputed through the oracle's CSR matrix, orthonormality;
* the n-state subspace angle bound from the oracle's gap;
* the mixed-precision solver against the plain one (same tolerance).
"""
import os

import numpy as np
import pytest
import torch

import inputs
from oracle import kp
from tests.metrics import subspace_sin_angle

pytestmark = pytest.mark.gpu

SOLVE = dict(n_states=16, block_m=24, degree=120, tol=1e-10, seed=1)
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "c2_evals.txt")
GOLDEN_MID = os.path.join(os.path.dirname(__file__), "golden", "c2mid_evals.txt")


def _golden(path=GOLDEN):
    rows = [l.split() for l in open(path) if not l.startswith("#")]
    return np.array([float(r[1]) for r in rows]), np.array([float(r[2]) for r in rows])


@pytest.fixture(scope="module")
def c2mid(khp):
    """The 160x48x48 workload's fields cut to the central 64x24x24 points
    (221184 unknowns), solved in the bench's launch configuration, with the
    oracle's eigenvectors (ARPACK, a few minutes on the host)."""
    from oracle import eig
    p = inputs.crop(inputs.config2(), (64, 24, 24))
    g = khp.KPGrid.from_problem(p)
    w, v = eig.lowest_arpack(kp.assemble(p), 17)
    yield p, g, w, v
    g.close()


@pytest.mark.parametrize("kw", [dict(), dict(degree=200, precision=2)])
def test_c2mid_eigenpairs_vs_oracle(c2mid, kw):
    """Eigenvalues against the stored oracle values (|dE| <= 1e-10 eV) and
    the largest principal angle of the 16-state subspace against the
    oracle's eigenvectors (<= 1e-7), plain FP64 and defect-corrected FP32
    filter."""
    p, g, w, v = c2mid
    r = g.eigensolve(**dict(SOLVE, **kw))
    assert r.stats["converged"] == 16
    ws, _ = _golden(GOLDEN_MID)
    assert np.abs(ws[:17] - w).max() <= 1e-12          # the stored values are this oracle's
    assert np.abs(r.evals - ws[:16]).max() <= 1e-10, np.abs(r.evals - ws[:16])
    assert ws[16] - ws[15] > 1e-6                       # n = 16 cuts no cluster
    sin = subspace_sin_angle(v[:, :16], r.evecs.cpu().numpy())
    assert sin <= 1e-7, sin


@pytest.fixture(scope="module")
def c2(khp):
    p = inputs.config2()
    g = khp.KPGrid.from_problem(p)
    r = g.eigensolve(**SOLVE)
    yield p, g, r
    g.close()


def test_c2_eigenvalues_vs_stored_oracle(c2):
    p, g, r = c2
    if not os.path.exists(GOLDEN):
        pytest.skip("stored oracle eigenvalues for the 2.21M-unknown grid not generated")
    w, wres = _golden()
    assert r.stats["converged"] == 16
    # |dE| <= 1e-10 eV plus the oracle's own error bound (res^2 / gap, tiny)
    assert np.abs(r.evals - w[:16]).max() <= 1e-10, np.abs(r.evals - w[:16])


def test_c2_residuals_through_oracle_csr(c2):
    p, g, r = c2
    H = kp.assemble(p)
    V = r.evecs.cpu().numpy()
    res = np.linalg.norm(H @ V - V * r.evals[None, :], axis=0)
    assert res.max() <= 2e-10, res
    G = V.conj().T @ V
    assert np.abs(G - np.eye(16)).max() < 1e-12
    # Rayleigh quotients through the oracle equal the returned eigenvalues
    rq = np.real(np.einsum("ij,ij->j", V.conj(), H @ V))
    assert np.abs(rq - r.evals).max() <= 1e-12
    # largest principal angle to the exact 16-state subspace <= ||R|| / gap
    if not os.path.exists(GOLDEN):
        return
    w, _ = _golden()
    gap = w[16] - r.evals[15]
    assert gap > 0
    bound = np.linalg.norm(H @ V - V * r.evals[None, :], 2) / gap
    assert bound <= 1e-6, bound


@pytest.mark.parametrize("kw", [dict(), dict(degree=200, precision=2)])
def test_c2_subspace_angle_bound_below_1e7(khp, kw):
    """At 2.21M unknowns: with the residual tolerance one decade below the
    bench's, the Davis-Kahan bound sin(theta) <= ||H V - V diag(E)||_2 / gap
    on the largest principal angle to the exact 16-state subspace (gap from
    the stored oracle's 17th eigenvalue, 1.1 meV above the 16th) is
    <= 1e-7, and the eigenvalues match the stored oracle to 1e-10 eV; plain
    FP64 and the defect-corrected FP32 filter."""
    if not os.path.exists(GOLDEN):
        pytest.skip("stored oracle eigenvalues for the 2.21M-unknown grid not generated")
    p = inputs.config2()
    g = khp.KPGrid.from_problem(p)
    r = g.eigensolve(**dict(SOLVE, tol=1e-11, **kw))
    w, _ = _golden()
    assert np.abs(r.evals - w[:16]).max() <= 1e-10
    H = kp.assemble(p)
    V = r.evecs.cpu().numpy()
    bound = np.linalg.norm(H @ V - V * r.evals[None, :], 2) / (w[16] - r.evals[15])
    assert bound <= 1e-7, bound
    g.close()


@pytest.mark.parametrize("kw", [dict(degree=80, precision=1, refine_sweeps=-1),
                                dict(degree=200, precision=2)])
def test_c2_mixed_precision_matches_plain(c2, kw):
    p, g, r = c2
    rm = g.eigensolve(**dict(SOLVE, **kw))
    assert rm.stats["launches_fp32"] >= 1
    assert np.abs(rm.evals - r.evals).max() <= 1e-10
    U, Vm = r.evecs, rm.evecs
    R = Vm - U @ (U.conj().T @ Vm)
    sin_max = torch.linalg.matrix_norm(R, ord=2).item()
    assert sin_max <= 1e-7, sin_max


def test_c5_gradients_full_size(khp):
    """Config 5 (200x64x64, 4.9M unknowns, B = 0): the Hellmann-Feynman
    gradients of L = (E2+E3)/2 - (E0+E1)/2 + sum_{i<8} E_i (doublet reading)
    with respect to V(r), the strain field and five gate levers.
    * kernel vs the oracle's HF formula on the same eigenvectors;
    * central differences along 20 seeded smooth unit-RMS directions of V,
      3 strain directions and the 5 levers (warm-started solves).  The
      lowest doublets are tunnel-split by 12 ueV, so the doublet-gap term is
      linear only for steps well below that: dV = 1e-7 eV (central-difference
      error 4e-8 relative, measured; at 1e-5 eV it is 4e-4), strain 1e-8."""
    from oracle import observables
    p = inputs.config5()
    n, dev = 8, torch.device("cuda")
    g = khp.KPGrid(p.nx, p.ny, p.nz, p.h, p.material, p.rot)
    V0 = torch.from_numpy(p.V.reshape(-1)).to(dev)
    S0 = torch.zeros(6 * p.n_points, dtype=torch.float64, device=dev)
    lev = torch.from_numpy(p.levers.reshape(5, -1)).to(dev)
    kw = dict(n_states=n, block_m=16, degree=200, precision=2, tol=1e-11, seed=3)
    wts = np.ones(n)
    wts[0:2] -= 0.5
    wts[2:4] += 0.5

    def solve(V, S, alpha, warm=None):
        g.set_fields(V, S, lev, alpha, p.B, p.gauge)
        return g.eigensolve(**kw, warm_start=warm)

    r = solve(V0, S0, np.zeros(5))
    dV, dS, dA = g.backward(r.evecs, r.evals, wts, levers=lev)
    # kernel vs oracle formula on the same vectors
    Vh = r.evecs.cpu().numpy()
    oV, oS, oA = observables.hf_gradients(Vh, wts, p.material, p.rot, p.levers)
    assert np.abs(dV.cpu().numpy() - oV).max() <= 1e-12 * np.abs(oV).max()
    assert np.abs(dS.cpu().numpy().reshape(6, -1) - oS).max() <= 1e-12 * np.abs(oS).max()
    assert np.abs(dA - oA).max() <= 1e-12 * np.abs(oA).max()

    rng = np.random.Generator(np.random.PCG64(2024))
    d = 1e-7
    L = lambda rr: float(wts @ rr.evals)
    worst = 0.0
    for _ in range(20):
        u = torch.from_numpy(inputs.smooth_noise(rng, (p.nz, p.ny, p.nx)).reshape(-1)).to(dev)
        fd = (L(solve(V0 + d * u, S0, np.zeros(5), r.evecs)) - L(solve(V0 - d * u, S0, np.zeros(5), r.evecs))) / (2 * d)
        an = float((dV * u).sum())
        worst = max(worst, abs(fd - an) / max(1.0, abs(an)))
    for c in (0, 2, 5):
        u = torch.zeros(6, p.n_points, dtype=torch.float64, device=dev)
        u[c] = torch.from_numpy(inputs.smooth_noise(rng, (p.nz, p.ny, p.nx)).reshape(-1)).to(dev)
        u = u.reshape(-1)
        ds = 1e-8
        fd = (L(solve(V0, S0 + ds * u, np.zeros(5), r.evecs)) - L(solve(V0, S0 - ds * u, np.zeros(5), r.evecs))) / (2 * ds)
        an = float((dS * u).sum())
        worst = max(worst, abs(fd - an) / max(1.0, abs(an)))
    for k in range(5):
        e = np.zeros(5)
        e[k] = d
        fd = (L(solve(V0, S0, e, r.evecs)) - L(solve(V0, S0, -e, r.evecs))) / (2 * d)
        worst = max(worst, abs(fd - dA[k]) / max(1.0, abs(dA[k])))
    assert worst <= 1e-6, worst
    g.close()


def test_c2_g_tensors_predict_zeeman_splitting(khp):
    """g-tensors at full size (the bench's g-tensor configuration): the
    g-matrix of the lowest doublet, from the response projections at
    B = +-0.01 T, predicts the splitting mu_B b |g n| of the two lowest
    states that the eigensolver finds at B = b n (b = 0.02 T, two
    directions), to the order-b^3 and solver-tolerance terms; the projected
    position pairs up (Kramers) on the two doublets."""
    from paper_2607_08447_b300.gtensor import MU_B, g_tensors
    p = inputs.config2()
    g = khp.KPGrid.from_problem(p)
    kw = dict(block_m=12, degree=200, precision=2, tol=1e-11, seed=1)
    r = g_tensors(g, solve_kw=kw)
    w = np.linalg.eigvalsh(r.position)
    assert abs(w[1] - w[0]) <= 1e-5 and abs(w[3] - w[2]) <= 1e-5
    b = 0.02
    for n in (np.array([1.0, 0.0, 0.0]), np.array([0.3, -0.5, 0.8]) / np.linalg.norm([0.3, -0.5, 0.8])):
        g.set_B(b * n)
        s = g.eigensolve(4, **kw)
        split = (s.evals[1] - s.evals[0]) / (MU_B * b)
        pred = np.linalg.norm(r.g_bonding @ n)
        assert abs(split - pred) <= 1e-4 * max(1.0, pred), (n, split, pred)
    g.close()


@pytest.fixture(scope="module")
def c2_h0_csr():
    p = inputs.config2()
    return p, kp.assemble_h0(p.with_(B=np.zeros(3)))


@pytest.mark.parametrize("kw", [dict(degree=120, precision=0), dict(degree=200, precision=2)])
def test_c2_h0_residuals_through_oracle_csr(khp, c2_h0_csr, kw):
    """The spin-independent H0 (1.1M unknowns at the C2 grid and fields, the
    CI orbital basis) in the bench's plain and defect-corrected settings:
    residuals and Rayleigh quotients through the oracle's CSR H0,
    orthonormality."""
    p, H = c2_h0_csr
    g = khp.KPGrid.from_problem(p, bands=3)
    r = g.eigensolve(16, block_m=24, tol=1e-10, seed=1, **kw)
    V = r.evecs.cpu().numpy()
    res = np.linalg.norm(H @ V - V * r.evals[None, :], axis=0)
    assert res.max() <= 2e-10, res
    assert np.abs(V.conj().T @ V - np.eye(16)).max() < 1e-12
    rq = np.real(np.einsum("ij,ij->j", V.conj(), H @ V))
    assert np.abs(rq - r.evals).max() <= 1e-12
    g.close()


def test_c2_filter_steps_sampled_against_oracle_rows(khp):
    """The two stencil kernels in the bench's launch configuration at full
    size (2.21M unknowns, 24 columns): the defect-corrected FP32 step of the
    plane-marching kernel (y = alpha H x + beta x + gamma prev + c_col src)
    and the FP64 apply of the per-point kernel, checked on 3000 sampled rows
    against the oracle's CSR rows applied to the same inputs in FP64."""
    p = inputs.config2()
    g = khp.KPGrid.from_problem(p)
    H = kp.assemble(p).tocsr()
    N, ld = p.n_unknowns, 24
    rng = np.random.default_rng(77)
    rows = np.sort(rng.choice(N, 3000, replace=False))
    Hs = H[rows]
    gen = torch.Generator(device="cuda").manual_seed(5)
    x, prev, src = (torch.randn((N, ld), dtype=torch.complex64, device="cuda", generator=gen) for _ in range(3))
    y = torch.zeros((N, ld), dtype=torch.complex64, device="cuda")
    coef = np.linspace(-0.7, 0.9, ld)
    al, be, ga = 0.41, -0.63, -0.37
    g.filter_step(x, y, al, be, ga, prev=prev, src=src, src_coef=coef)
    xd = x.cpu().numpy().astype(np.complex128)
    ref = (al * (Hs @ xd) + be * xd[rows] + ga * prev.cpu().numpy()[rows].astype(np.complex128)
           + src.cpu().numpy()[rows].astype(np.complex128) * coef)
    got = y.cpu().numpy()[rows].astype(np.complex128)
    scale = np.abs(al * (Hs @ xd)).max() + np.abs(xd).max() + 2 * np.abs(prev.cpu().numpy()).max()
    assert np.abs(got - ref).max() <= 2e-6 * scale
    del x, prev, src, y
    X = torch.randn((N, ld), dtype=torch.complex128, device="cuda", generator=gen)
    Y = g.apply(X, precision=0)
    refd = Hs @ X.cpu().numpy()
    assert np.abs(Y.cpu().numpy()[rows] - refd).max() <= 1e-13 * np.abs(refd).max()
    g.close()


def test_c4_batched_residuals_through_oracle_csr(khp):
    """Two points of the 64-point sweep at full size (the bench's
    batched configuration: grouped filter launches, defect-corrected FP32
    filter, degree 200, block width 16, tol 1e-10 eV): residuals and
    Rayleigh quotients of the 12 returned states through the oracle's CSR
    matrices, orthonormality."""
    probs = inputs.config4()[:2]
    grids = [khp.KPGrid.from_problem(q) for q in probs]
    rs = khp.solve_batched(grids, 12, block_m=16, degree=200, precision=2, tol=1e-10, seed=1, graph=True,
                           grouped=True)
    for q, r in zip(probs, rs):
        H = kp.assemble(q)
        V = r.evecs.cpu().numpy()
        res = np.linalg.norm(H @ V - V * r.evals[None, :], axis=0)
        assert res.max() <= 2e-10, res
        assert np.abs(V.conj().T @ V - np.eye(12)).max() < 1e-12
        rq = np.real(np.einsum("ij,ij->j", V.conj(), H @ V))
        assert np.abs(rq - r.evals).max() <= 1e-12
    for gr in grids:
        gr.close()
