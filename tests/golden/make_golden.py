"""Writes the stored oracle eigenvalues used by the full-size GPU tests.

    python tests/golden/make_golden.py [c1] [c2]

Calls only the FP64 oracle (`oracle/`) on the seeded workloads of `inputs/`:
  c1_evals.txt  config 1 (10x8x8): lowest 10 eigenvalues, dense LAPACK
  c2_evals.txt  config 2 (160x48x48, 2.21M unknowns): lowest 17 eigenvalues,
                thick-restarted block Lanczos, residual tolerance 1e-11 eV
Each file records the generator, the method and the oracle residuals.
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import inputs  # noqa: E402
from oracle import eig, kp  # noqa: E402


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


def c2():
    p = inputs.config2()
    t0 = time.time()
    H = kp.assemble(p)
    t1 = time.time()
    w, v, res, cycles = eig.lowest_block_lanczos(H, 17, block=4, tol=1e-11, max_cycles=2000,
                                                 return_residuals=True)
    t2 = time.time()
    _write("c2_evals.txt", ["config 2 (inputs.config2), 160x48x48 h=0.5 nm, 2211840 unknowns, B=0.5 T",
                            "oracle: kp.assemble + eig.lowest_block_lanczos(block=4, tol=1e-11), FP64",
                            f"assembly {t1 - t0:.0f} s, solve {t2 - t1:.0f} s, {cycles} restart cycles",
                            "columns: index, eigenvalue [eV], oracle residual ||Hv - wv|| [eV]"], w, res)


if __name__ == "__main__":
    which = sys.argv[1:] or ["c1", "c2"]
    if "c1" in which:
        c1()
    if "c2" in which:
        c2()
