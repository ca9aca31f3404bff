"""Coarse-grid start of the eigensolve (khp_solver_opts.start = 1): the lowest
states of the grid of every second point at twice the spacing, prolongated
trilinearly, start the block.  Checked here: the converged eigenpairs equal
those of the random start and of the FP64 oracle (even and odd grid sizes,
both gauges, a point mask, plain and defect-corrected), the start block is
a good one (the residuals of the first Rayleigh-Ritz after the
prolongation far below those after a random start), and grids too small
for a coarse block fall back to the random start."""
import numpy as np
import pytest

import inputs
from oracle import eig, kp

pytestmark = pytest.mark.gpu

CASES = {
    "even_symmetric": dict(shape=(28, 18, 16), B=(0.5, 0.0, 0.0), gauge=0, rot="device", mask=False),
    "odd_landau": dict(shape=(27, 17, 15), B=(0.2, 0.3, 0.1), gauge=1, rot="identity", mask=False),
    "mask": dict(shape=(26, 16, 14), B=(0.1, 0.0, 0.2), gauge=0, rot="device", mask=True),
}


@pytest.mark.parametrize("case", list(CASES))
def test_coarse_start_matches_random_and_oracle(khp, case):
    c = CASES[case]
    p = inputs.small_problem(*c["shape"], h=0.5, seed=31, rot=c["rot"], B=c["B"], gauge=c["gauge"],
                             strain=True, mask=c["mask"])
    g = khp.KPGrid.from_problem(p)
    kw = dict(n_states=8, block_m=16, degree=40, tol=1e-10, seed=3)
    rr = g.eigensolve(**kw, start="random")
    rc = g.eigensolve(**kw, start="coarse")
    assert rr.stats["start_iterations"] == 0
    assert rc.stats["start_iterations"] > 0 and rc.stats["ms_start"] > 0
    assert rc.stats["converged"] == 8
    assert np.abs(rc.evals - rr.evals).max() <= 1e-10
    H = kp.assemble(p)
    w, _ = eig.lowest_arpack(H, 8, mask=p.mask)
    assert np.abs(rc.evals - w).max() <= 1e-9
    # the prolongated block: first residuals far below a random start's (a
    # random point mask, restricted by injection, leaves a coarse domain of
    # its own: there the start only has to beat a random one)
    bound = 1.0 if c["mask"] else 0.05
    assert rc.stats["res_history"][0] < bound * rr.stats["res_history"][0]


def test_coarse_start_defect_corrected(khp):
    p = inputs.small_problem(30, 16, 16, h=0.5, seed=32, rot="device", B=(0.5, 0.0, 0.0), gauge=0, strain=True)
    g = khp.KPGrid.from_problem(p)
    kw = dict(n_states=8, block_m=16, degree=60, tol=1e-10, seed=4, precision=2)
    rr = g.eigensolve(**kw, start="random")
    rc = g.eigensolve(**kw, start="coarse")
    assert rc.stats["start_iterations"] > 0
    assert np.abs(rc.evals - rr.evals).max() <= 1e-10
    V = rc.evecs.cpu().numpy()
    H = kp.assemble(p)
    res = np.linalg.norm(H @ V - V * rc.evals[None, :], axis=0)
    assert res.max() <= 1e-9


def test_coarse_start_follows_new_fields(khp):
    """A second solve after set_fields rebuilds the coarse fields: its
    eigenvalues follow the new potential."""
    p = inputs.small_problem(24, 16, 14, h=0.5, seed=33, B=(0.3, 0.0, 0.0))
    g = khp.KPGrid.from_problem(p)
    kw = dict(n_states=6, block_m=16, degree=40, tol=1e-10, seed=5)
    r0 = g.eigensolve(**kw, start="coarse")
    shift = 2e-3
    g.set_fields(p.V + shift, p.strain, None, None, p.B, p.gauge)
    r1 = g.eigensolve(**kw, start="coarse")
    assert np.abs((r1.evals - r0.evals) - shift).max() <= 1e-9


def test_coarse_start_falls_back_on_tiny_grids(khp):
    p = inputs.small_problem(5, 4, 4, h=1.0, seed=34)
    g = khp.KPGrid.from_problem(p)
    r = g.eigensolve(n_states=4, block_m=16, degree=20, tol=1e-10, seed=6, start="coarse")
    assert r.stats["start_iterations"] == 0
    assert r.stats["converged"] == 4
    w, _ = eig.lowest_dense(kp.assemble(p), 4)
    assert np.abs(r.evals - w).max() <= 1e-9


def test_coarse_start_spin_independent_h0(khp):
    """The three-band H0 handle takes the coarse-grid start as well."""
    p = inputs.small_problem(28, 16, 16, h=0.5, seed=35, rot="device", strain=True)
    g = khp.KPGrid.from_problem(p, bands=3)
    kw = dict(n_states=6, block_m=16, degree=40, tol=1e-10, seed=7)
    rr = g.eigensolve(**kw, start="random")
    rc = g.eigensolve(**kw, start="coarse")
    assert rc.stats["start_iterations"] > 0
    assert np.abs(rc.evals - rr.evals).max() <= 1e-10
    # a 14x8x8 coarse grid at 1 nm: a coarser start than on larger grids
    assert rc.stats["res_history"][0] < 0.2 * rr.stats["res_history"][0]


def test_block_output_restarts_a_solve(khp):
    """block_out receives the final orthonormal Ritz block: its first
    n_states columns are the returned eigenvectors; a solve of a slightly
    changed potential warm-started from the whole block needs fewer outer
    iterations than one from the coarse grid and finds the same levels as a
    cold solve (both vs the dense oracle)."""
    import torch
    p = inputs.small_problem(12, 8, 6, h=0.5, seed=3, strain=True)
    g = khp.KPGrid.from_problem(p)
    n, m = 8, 16
    blk = torch.empty((g.N, m), dtype=torch.complex128, device="cuda")
    kw = dict(block_m=m, degree=30, tol=1e-11, seed=2)
    r = g.eigensolve(n, block_out=blk, start="coarse", **kw)
    X = blk.cpu().numpy()
    assert np.abs(X[:, :n] - r.evecs.cpu().numpy()).max() == 0.0
    assert np.abs(X.conj().T @ X - np.eye(m)).max() <= 1e-12
    V2 = p.V + 1e-3 * inputs.smooth_noise(np.random.default_rng(8), p.V.shape)
    g.set_fields(V2, p.strain, None, None, p.B, p.gauge)
    warm = g.eigensolve(n, warm_start=blk.clone(), **kw)
    cold = g.eigensolve(n, start="coarse", **kw)
    ref, _ = eig.lowest_dense(kp.assemble(p.with_(V=V2)), n)
    assert np.abs(warm.evals - ref).max() <= 1e-10
    assert np.abs(cold.evals - ref).max() <= 1e-10
    assert warm.stats["iterations"] < cold.stats["iterations"]
    with pytest.raises(ValueError):
        g.eigensolve(n, block_out=torch.empty((g.N, m - 2), dtype=torch.complex128, device="cuda"), **kw)
    g.close()
