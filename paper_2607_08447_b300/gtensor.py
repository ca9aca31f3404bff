"""g-matrices of the two lowest Kramers doublets of a double dot and the
g-tensors of its left and right dots (Sec. III B: the g-tensors of Eq. 16
come from the g-matrix of the spin-mixed bonding and anti-bonding states).

Grid-sized work runs in the library: the B = 0 eigensolve of the 6x6
operator, the operator applies at B = +-d e_j, the projections of those
applies on the states (khp_project, tensor cores) and the position moments
(khp_position_moments).  The host handles 4 x 4 matrices only.

g-matrix of a doublet with coefficient block c ([4][2]) in the basis of
the four states U:  M_j = U^H (H(d e_j) - H(-d e_j)) U / (2 d) is the
response to B_j (Zeeman plus the orbital part through the Peierls phases),
c^H M_j c = (mu_B / 2) sum_i g_ij sigma_i defines g.

Left/right dots: the projected position along the dot axis, X4 = U^H x U,
is time-reversal even on the four-dimensional span of the two doublets, so
its eigenvalues pair up; the eigenvectors of the lower pair span the left
dot's doublet, those of the upper pair the right dot's.  The symmetric
g-tensor of a dot is sign(det g) (g^T g)^(1/2).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

MU_B = 5.7883818060e-5          # Bohr magneton, eV / T


def _pauli(P):
    """Vector part (a_x, a_y, a_z) of the Hermitian 2x2 P = a_0 + a.sigma."""
    return np.array([P[0, 1].real, -P[0, 1].imag, 0.5 * (P[0, 0].real - P[1, 1].real)])


def g_matrix_of(M, c):
    """g-matrix (3x3) of the doublet c ([m][2]) from the responses M [3][m][m]."""
    P = np.einsum("ai,jab,bk->jik", c.conj(), M, c)          # [3][2][2]
    return np.stack([_pauli(P[j]) for j in range(3)], axis=1) * (2.0 / MU_B)


def symmetric_g(g):
    """sign(det g) (g^T g)^(1/2), the symmetric polar factor of g."""
    w, v = np.linalg.eigh(g.T @ g)
    return np.sign(np.linalg.det(g)) * (v @ np.diag(np.sqrt(np.maximum(w, 0.0))) @ v.T)


@dataclass
class GTensorResult:
    energies: np.ndarray        # the four lowest energies at B = 0 (eV)
    delta: float                # bonding / anti-bonding separation (eV)
    tunnel: float               # t = delta / sqrt(2) (eV)
    response: np.ndarray        # [3][4][4] U^H dH/dB_j U (eV / T)
    position: np.ndarray        # [4][4] U^H x_axis U (nm)
    g_bonding: np.ndarray
    g_antibonding: np.ndarray
    g_left: np.ndarray
    g_right: np.ndarray
    gsym_left: np.ndarray
    gsym_right: np.ndarray


def g_tensors(grid, delta_b=1e-2, axis=0, solve_kw=None, states=None):
    """g-matrices of the double dot held by `grid` (6-band handle, fields
    set; its field B is set to zero for the solve and restored after).
    `states` = (E, U) skips the eigensolve (U: complex128 [N][4] on the
    device, the four lowest states at B = 0)."""
    if getattr(grid, "bands", 6) != 6:
        raise ValueError("g-matrices need the 6-band operator")
    if not delta_b > 0:
        raise ValueError("delta_b must be positive")
    B0 = np.array(grid.B, dtype=np.float64)
    try:
        grid.set_B(np.zeros(3))
        if states is None:
            kw = dict(block_m=16, degree=40, tol=1e-11, seed=1)
            kw.update(solve_kw or {})
            r = grid.eigensolve(4, **kw)
            E, U = np.asarray(r.evals), r.evecs
        else:
            E, U = np.asarray(states[0], dtype=np.float64), states[1]
        M = np.zeros((3, 4, 4), dtype=np.complex128)
        for j in range(3):
            e = np.zeros(3)
            e[j] = delta_b
            grid.set_B(e)
            _, Sp = grid.project(U, grid.apply(U))
            grid.set_B(-e)
            _, Sm = grid.project(U, grid.apply(U))
            M[j] = (Sp - Sm) / (2.0 * delta_b)
    finally:
        grid.set_B(B0)
    X4 = grid.position_moments(U)[axis]
    _, v = np.linalg.eigh(X4)
    cL, cR = v[:, :2], v[:, 2:]
    I4 = np.eye(4)
    gL, gR = g_matrix_of(M, cL), g_matrix_of(M, cR)
    delta = 0.5 * (E[2] + E[3] - E[0] - E[1])
    return GTensorResult(E, float(delta), float(delta / np.sqrt(2.0)), M, X4,
                         g_matrix_of(M, I4[:, :2]), g_matrix_of(M, I4[:, 2:]), gL, gR,
                         symmetric_g(gL), symmetric_g(gR))
