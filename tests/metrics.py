"""Comparison metrics shared by the tests (no method arithmetic)."""
import numpy as np


def subspace_sin_angle(U, V):
    """sin of the largest principal angle between span(U) and span(V), for
    orthonormal columns: ||V - U U^H V||_2 (accurate for tiny angles)."""
    R = V - U @ (U.conj().T @ V)
    return float(np.linalg.norm(R, 2))


def clusters(w, sep=1e-6):
    """Split ascending eigenvalues into clusters separated by more than sep."""
    out, cur = [], [0]
    for i in range(1, len(w)):
        if w[i] - w[i - 1] > sep:
            out.append(cur)
            cur = [i]
        else:
            cur.append(i)
    out.append(cur)
    return out
