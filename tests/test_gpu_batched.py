"""Batched sweep solver (khp_eigensolve_batched) against single solves and
the dense oracle: uneven grids, different fields per sweep point, with and
without CUDA-graph rounds, and with the block-width autotuner."""
import numpy as np
import pytest

import inputs
from oracle import eig, kp

pytestmark = pytest.mark.gpu


def _sweep(count=5):
    out = []
    shapes = [(11, 7, 6), (9, 8, 7), (13, 6, 6), (10, 7, 7), (12, 6, 5), (8, 8, 8)]
    for k in range(count):
        nx, ny, nz = shapes[k % len(shapes)]
        out.append(inputs.small_problem(nx, ny, nz, h=0.6, seed=40 + k, rot="identity" if k % 2 else "device",
                                        B=(0.2 * k, 0.0, 0.0), strain=bool(k % 2)))
    return out


@pytest.mark.parametrize("graph", [True, False])
def test_batched_matches_oracle(khp, graph):
    probs = _sweep(5)
    grids = [khp.KPGrid.from_problem(p) for p in probs]
    rs = khp.solve_batched(grids, 8, block_m=16, degree=20, tol=1e-10, graph=graph)
    for p, r in zip(probs, rs):
        w, _ = eig.lowest_dense(kp.assemble(p), 8)
        assert np.abs(r.evals - w).max() <= 1e-10
        V = r.evecs.cpu().numpy()
        assert np.abs(V.conj().T @ V - np.eye(8)).max() < 1e-12
        assert r.stats["batch_rounds"] >= r.stats["iterations"]
        if graph:
            assert r.stats["batch_graphs"] >= 1


def test_batched_equals_single_solves(khp):
    probs = _sweep(4)
    grids = [khp.KPGrid.from_problem(p) for p in probs]
    rb = khp.solve_batched(grids, 8, block_m=16, degree=20, tol=1e-10, graph=True)
    for g, r in zip(grids, rb):
        r1 = g.eigensolve(8, block_m=16, degree=20, tol=1e-10)
        assert np.abs(r1.evals - r.evals).max() <= 1e-11


def test_batched_mixed_and_autotune(khp):
    probs = _sweep(3)
    grids = [khp.KPGrid.from_problem(p) for p in probs]
    rs = khp.solve_batched(grids, 8, degree=20, precision=1, refine_sweeps=-1, tol=1e-10, autotune=True)
    chosen = {r.stats["block_m"] for r in rs}
    assert len(chosen) == 1 and chosen.pop() in (12, 16, 20)
    assert sum(r.stats["autotune_ms"] > 0 for r in rs) == 1
    for p, r in zip(probs, rs):
        w, _ = eig.lowest_dense(kp.assemble(p), 8)
        assert np.abs(r.evals - w).max() <= 1e-10


@pytest.mark.parametrize("graph", [True, False])
def test_batched_grouped_filter_launches(khp, graph):
    """Defect-corrected FP32 filter (precision 2) with one grouped launch per
    filter step across the problems (KHP_BATCH_GROUPED; the B = 0 point and
    the B != 0 points go out in separate groups): eigenvalues equal to the
    ungrouped batch and to the dense oracle."""
    probs = _sweep(5)
    grids = [khp.KPGrid.from_problem(p) for p in probs]
    kw = dict(block_m=16, degree=40, precision=2, tol=1e-10)
    rg = khp.solve_batched(grids, 8, graph=graph, grouped=True, **kw)
    ru = khp.solve_batched(grids, 8, graph=graph, grouped=False, **kw)
    for p, a, b in zip(probs, rg, ru):
        assert np.abs(a.evals - b.evals).max() <= 1e-14
        w, _ = eig.lowest_dense(kp.assemble(p), 8)
        assert np.abs(a.evals - w).max() <= 1e-10
        V = a.evecs.cpu().numpy()
        assert np.abs(V.conj().T @ V - np.eye(8)).max() < 1e-12


def test_batched_rejects_bad_input(khp):
    probs = _sweep(2)
    grids = [khp.KPGrid.from_problem(p) for p in probs]
    with pytest.raises(khp.KHPError):
        khp.solve_batched([grids[0], grids[0]], 8, block_m=16)


def test_batched_coarse_start(khp):
    """start = 'coarse' in a batched call: the coarse grids of the eligible
    problems are solved together and prolongated; a grid too small for a
    coarse block starts from a random one.  Plain and grouped
    defect-corrected rounds; eigenvalues equal to single random-start solves
    and to the oracle."""
    shapes = [(20, 12, 10), (16, 14, 12), (18, 10, 12), (5, 4, 4)]
    probs = [inputs.small_problem(*sh, h=0.5, seed=60 + k, rot="device", B=(0.3 + 0.1 * k, 0.0, 0.1), strain=True)
             for k, sh in enumerate(shapes)]
    grids = [khp.KPGrid.from_problem(p) for p in probs]
    rc = None
    for grouped, prec in ((False, 0), (True, 2)):
        kw = dict(block_m=16, degree=40, precision=prec, tol=1e-10)
        rc = khp.solve_batched(grids, 8, graph=True, grouped=grouped, start="coarse", **kw)
        for k, (g, r) in enumerate(zip(grids, rc)):
            r1 = g.eigensolve(8, start="random", **kw)
            assert np.abs(r1.evals - r.evals).max() <= 1e-10
            if k < 3:
                assert r.stats["start_iterations"] > 0
            else:
                assert r.stats["start_iterations"] == 0
    w, _ = eig.lowest_arpack(kp.assemble(probs[0]), 8)
    assert np.abs(rc[0].evals - w).max() <= 1e-9
