"""Writes the stored oracle eigenvalues used by the full-size GPU tests.

    python tests/golden/make_golden.py [c1] [c2mid] [c2]

Calls only the FP64 oracle (`oracle/`) on the seeded workloads of `inputs/`:
  c1_evals.txt     config 1 (10x8x8): lowest 10 eigenvalues, dense LAPACK
  c2mid_evals.txt  the 160x48x48 workload's fields cut to its central
                   64x24x24 points (221184 unknowns, B = 0.5 T): lowest 18
                   eigenvalues, ARPACK (oracle.eig.lowest_arpack)
  c2_evals.txt     config 2 (160x48x48, 2.21M unknowns, B = 0.5 T): lowest 18
                   eigenvalues, ARPACK (oracle.eig.lowest_arpack)
Each file records the generator, the method, the run time and the oracle
residuals ||H v - w v|| recomputed from the assembled matrix.  At B != 0 no
level is exactly degenerate, which the single-vector ARPACK path needs.
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import inputs  # noqa: E402
from oracle import eig, kp  # noqa: E402

C2MID = (64, 24, 24)


def _write(name, header, w, res):
    with open(os.path.join(HERE, name), "w") as fh:
        for line in header:
            fh.write("# " + line + "\n")
        for i, (e, r) in enumerate(zip(w, res)):
            fh.write(f"{i:3d} {e:.17e} {r:.3e}\n")


def c1():
    p = inputs.config1()
    H = kp.assemble(p)
    w, v = eig.lowest_dense(H, 10)
    res = np.linalg.norm(H @ v - v * w[None, :], axis=0)
    _write("c1_evals.txt", ["config 1 (inputs.config1), 10x8x8 h=1 nm, 3840 unknowns",
                            "oracle: kp.assemble + eig.lowest_dense (LAPACK evr), FP64",
                            "columns: index, eigenvalue [eV], oracle residual ||Hv - wv|| [eV]"], w, res)


def _arpack(p, name, title, n=18, ncv=None):
    t0 = time.time()
    H = kp.assemble(p)
    t1 = time.time()
    w, v, res, nmv = eig.lowest_arpack(H, n, tol=1e-13, ncv=ncv, return_residuals=True)
    t2 = time.time()
    _write(name, [title,
                  "oracle: kp.assemble + eig.lowest_arpack (SciPy eigsh, which='SA', tol=1e-13), FP64",
                  f"assembly {t1 - t0:.0f} s, solve {t2 - t1:.0f} s, {nmv} products H x, {os.cpu_count()} host cores",
                  "columns: index, eigenvalue [eV], oracle residual ||Hv - wv|| [eV]"], w, res)


def c2mid():
    p = inputs.crop(inputs.config2(), C2MID)
    _arpack(p, "c2mid_evals.txt",
            f"config 2 fields (inputs.config2) cut to the central {C2MID[0]}x{C2MID[1]}x{C2MID[2]} points "
            f"(inputs.crop), h=0.5 nm, {p.n_unknowns} unknowns, B=0.5 T", ncv=80)


def c2():
    p = inputs.config2()
    _arpack(p, "c2_evals.txt",
            f"config 2 (inputs.config2), 160x48x48 h=0.5 nm, {p.n_unknowns} unknowns, B=0.5 T", ncv=120)


if __name__ == "__main__":
    which = sys.argv[1:] or ["c1", "c2mid", "c2"]
    for name in ("c1", "c2mid", "c2"):
        if name in which:
            globals()[name]()
