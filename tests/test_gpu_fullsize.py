"""Full-size checks on the 160x48x48 workload (2.21M unknowns) in the launch
configuration bench.py times (16 states, block 24, degree 120, tol 1e-10 eV).

* eigenvalues against the stored FP64 oracle values (block Lanczos, written
  by tests/golden/make_golden.py, which calls only the oracle);
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

pytestmark = pytest.mark.gpu

SOLVE = dict(n_states=16, block_m=24, degree=120, tol=1e-10, seed=1)
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "c2_evals.txt")


def _golden():
    rows = [l.split() for l in open(GOLDEN) if not l.startswith("#")]
    return np.array([float(r[1]) for r in rows]), np.array([float(r[2]) for r in rows])


@pytest.fixture(scope="module")
def c2(khp):
    p = inputs.config2()
    g = khp.KPGrid.from_problem(p)
    r = g.eigensolve(**SOLVE)
    yield p, g, r
    g.close()


def test_c2_eigenvalues_vs_stored_oracle(c2):
    p, g, r = c2
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
    w, _ = _golden()
    gap = w[16] - r.evals[15]
    assert gap > 0
    bound = np.linalg.norm(H @ V - V * r.evals[None, :], 2) / gap
    assert bound <= 1e-6, bound


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
