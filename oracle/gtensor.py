"""FP64 oracle of the g-matrices of the double dot (Sec. III B: the g-tensors
of Eq. 16 are built from the g-matrix of the spin-mixed bonding and
anti-bonding single-particle states).  Test infrastructure only.

g-matrix of a Kramers doublet.  For a doublet spanned by the columns of
U ([N][2]) of H at B = 0, the magnetic response is M_j = dH/dB_j at B = 0
(Zeeman term plus the orbital response through the Peierls phases), taken
by central differences of the assembled operator,
    M_j = (H(+d e_j) - H(-d e_j)) / (2 d).
Its projection P_j = U^H M_j U is written (mu_B / 2) sum_i g_ij sigma_i
(the trace vanishes by time reversal), which defines g.  The g-tensor
G = g^T g does not depend on the basis chosen inside the doublet; the
squared principal g-factors are its eigenvalues, and the Zeeman splitting
in a field B is mu_B |g B|.

Left and right dots (a reading: the paper builds g_L and g_R from the
bonding and anti-bonding states without saying how).  The lowest two
Kramers doublets of the double dot (bonding, anti-bonding) span a
four-dimensional space closed under time reversal.  The position along the
dot axis x, projected on it (X4 = U^H x U), is time-reversal even, so its
eigenvalues come in degenerate pairs: the lower pair spans the left-dot
doublet, the upper pair the right-dot doublet.  g_L and g_R are the
g-matrices of those doublets (the response matrices M_j rotated into the
localised basis), and the symmetric g-tensor of each is
    g_sym = sign(det g) (g^T g)^(1/2),
the symmetric factor of the polar decomposition of g with the sign of
det g (the one property of g, besides G, that no change of doublet basis
alters).
"""
from __future__ import annotations

import numpy as np

from . import eig, kp

MU_B = kp.MU_B


def pauli_components(P):
    """(a_x, a_y, a_z) of a Hermitian 2x2 matrix P = a_0 1 + a . sigma."""
    return np.array([P[0, 1].real, -P[0, 1].imag, 0.5 * (P[0, 0] - P[1, 1]).real])


def lowest_states(prob, n):
    """The lowest n eigenpairs of the 6x6 operator at B = 0 (dense)."""
    p0 = prob.with_(B=np.zeros(3))
    return eig.lowest_dense(kp.assemble(p0), n, mask=prob.mask)


def magnetic_response(prob, U, delta_b=1e-2):
    """[3][m][m] matrices U^H M_j U, M_j the central difference of H(B)
    about B = 0 along e_j."""
    m = U.shape[1]
    out = np.zeros((3, m, m), dtype=complex)
    for j in range(3):
        e = np.zeros(3)
        e[j] = delta_b
        Hp = kp.assemble(prob.with_(B=e))
        Hm = kp.assemble(prob.with_(B=-e))
        out[j] = U.conj().T @ ((Hp - Hm) @ U) / (2.0 * delta_b)
    return out


def g_matrix(M, c=None):
    """g-matrix of the doublet c ([m][2] coefficients in the basis of the
    response matrices M [3][m][m]; default: the first two basis states)."""
    if c is None:
        c = np.eye(M.shape[1])[:, :2]
    g = np.zeros((3, 3))
    for j in range(3):
        g[:, j] = 2.0 / MU_B * pauli_components(c.conj().T @ M[j] @ c)
    return g


def g_tensor(g):
    """G = g^T g and the principal g-factors (ascending)."""
    G = g.T @ g
    return G, np.sqrt(np.clip(np.linalg.eigvalsh(G), 0.0, None))


def symmetric_g(g):
    """sign(det g) (g^T g)^(1/2)."""
    w, v = np.linalg.eigh(g.T @ g)
    S = (v * np.sqrt(np.clip(w, 0.0, None))) @ v.T
    return np.sign(np.linalg.det(g)) * S


def position_matrix(prob, U, axis=0):
    """U^H x_axis U, x_axis the grid coordinate (nm) along `axis`, centred."""
    n = (prob.nx, prob.ny, prob.nz)[axis]
    x1 = (np.arange(n) - 0.5 * (n - 1)) * prob.h
    if axis == 0:
        x = np.broadcast_to(x1[None, None, :], (prob.nz, prob.ny, prob.nx))
    elif axis == 1:
        x = np.broadcast_to(x1[None, :, None], (prob.nz, prob.ny, prob.nx))
    else:
        x = np.broadcast_to(x1[:, None, None], (prob.nz, prob.ny, prob.nx))
    w = np.repeat(x.reshape(-1), 6)          # unknown 6 p + b sits at point p
    return U.conj().T @ (w[:, None] * U)


def localised_doublets(X4):
    """Coefficients (c_L, c_R), [4][2] each, of the left and right doublets:
    the eigenvectors of the projected position for its lower and upper
    eigenvalue pair."""
    w, v = np.linalg.eigh(X4)
    return v[:, :2], v[:, 2:]


def dqd_g_tensors(prob, delta_b=1e-2, axis=0):
    """Bonding/anti-bonding energies, their g-matrices, and the g-matrices
    and symmetric g-tensors of the localised left and right doublets."""
    E, U = lowest_states(prob, 4)
    M = magnetic_response(prob, U, delta_b)
    cL, cR = localised_doublets(position_matrix(prob, U, axis))
    I4 = np.eye(4)
    gb, ga = g_matrix(M, I4[:, :2]), g_matrix(M, I4[:, 2:])
    gL, gR = g_matrix(M, cL), g_matrix(M, cR)
    return dict(E=E, delta=0.5 * (E[2] + E[3] - E[0] - E[1]), g_bonding=gb, g_antibonding=ga,
                g_left=gL, g_right=gR, gsym_left=symmetric_g(gL), gsym_right=symmetric_g(gR), M=M)
