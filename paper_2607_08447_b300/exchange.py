"""Magnetic two-hole model and anisotropic exchange of the double dot
(Sec. III B, Eqs. 16-17): host arithmetic on 3x3 and 5x5 matrices,
vectorised over field directions.

* Eq. 16 in the basis {S(0,2), S(1,1), T+(1,1), T-(1,1), T0(1,1)} with
  bbar = mu_B (R(-theta_so) g_L + R(theta_so) g_R) B / 2 and
  db = mu_B (R(-theta_so) g_L - R(theta_so) g_R) B / 2;
* t = Delta / sqrt(2); U - eps = 2 t^2 / J for the exchange J of the CI;
* Eq. 17: Jhat = J R(-2 theta_so), Jt = R_L Jhat R_R^T,
  |J_perp| = |(Jt_xx + Jt_yy) + i (Jt_xy - Jt_yx)| / 2, J_par = Jt_zz;
  delta E_Z = |db|.
R(a) rotates by the angle a about n_so; R_L carries n_L = g_L B / |g_L B|
onto z along the shortest arc (likewise R_R), so Jt_zz = n_L . Jhat n_R.
"""
from __future__ import annotations

import numpy as np

MU_B = 5.7883818060e-5          # eV / T


def axis_rotation(n, angle):
    """Rotation matrices by `angle` (scalar or array [...]) about the unit
    axis n ([3] or [...][3]); returns [...][3][3]."""
    n = np.asarray(n, dtype=np.float64)
    n = n / np.linalg.norm(n, axis=-1, keepdims=True)
    angle = np.asarray(angle, dtype=np.float64)
    shape = np.broadcast_shapes(n.shape[:-1], angle.shape)
    n = np.broadcast_to(n, shape + (3,))
    c = np.cos(angle)[..., None, None]
    s = np.sin(angle)[..., None, None]
    K = np.zeros(shape + (3, 3))
    K[..., 0, 1], K[..., 0, 2] = -n[..., 2], n[..., 1]
    K[..., 1, 0], K[..., 1, 2] = n[..., 2], -n[..., 0]
    K[..., 2, 0], K[..., 2, 1] = -n[..., 1], n[..., 0]
    return c * np.eye(3) + s * K + (1.0 - c) * np.einsum("...i,...j->...ij", n, n)


def to_z(n):
    """Shortest-arc rotations carrying the unit vectors n ([...][3]) onto z."""
    n = np.asarray(n, dtype=np.float64)
    n = n / np.linalg.norm(n, axis=-1, keepdims=True)
    ax = np.stack([n[..., 1], -n[..., 0], np.zeros_like(n[..., 0])], axis=-1)    # n x z
    s = np.linalg.norm(ax, axis=-1)
    ang = np.arctan2(s, n[..., 2])
    safe = np.where(s[..., None] > 1e-15, ax, np.array([1.0, 0.0, 0.0]))
    return axis_rotation(safe, np.where(s > 1e-15, ang, np.where(n[..., 2] > 0, 0.0, np.pi)))


def zeeman_fields(gL, gR, theta_so, n_so, B):
    """(bbar, db), each [...][3] eV, for fields B [...][3] T."""
    B = np.asarray(B, dtype=np.float64)
    AL = axis_rotation(n_so, -theta_so) @ gL
    AR = axis_rotation(n_so, theta_so) @ gR
    bL = 0.5 * MU_B * np.einsum("ij,...j->...i", AL, B)
    bR = 0.5 * MU_B * np.einsum("ij,...j->...i", AR, B)
    return bL + bR, bL - bR


def hamiltonian_b(u_minus_eps, t, bbar, db):
    """Eq. 16 as [...][5][5] complex for bbar, db of shape [...][3]."""
    bbar = np.asarray(bbar, dtype=np.float64)
    db = np.asarray(db, dtype=np.float64)
    shape = np.broadcast_shapes(bbar.shape[:-1], db.shape[:-1])
    H = np.zeros(shape + (5, 5), dtype=np.complex128)
    s = 1.0 / np.sqrt(2.0)
    dp = (db[..., 0] + 1j * db[..., 1]) * s          # (db_x + i db_y) / sqrt2
    bp = (bbar[..., 0] + 1j * bbar[..., 1]) * s
    H[..., 0, 0] = u_minus_eps
    H[..., 0, 1] = H[..., 1, 0] = np.sqrt(2.0) * t
    H[..., 1, 2] = -dp
    H[..., 1, 3] = np.conj(dp)
    H[..., 1, 4] = db[..., 2]
    H[..., 2, 2] = bbar[..., 2]
    H[..., 3, 3] = -bbar[..., 2]
    H[..., 2, 4] = np.conj(bp)
    H[..., 3, 4] = bp
    # lower triangle by Hermiticity
    iu = np.triu_indices(5, 1)
    H[..., iu[1], iu[0]] = np.conj(H[..., iu[0], iu[1]])
    return H


def anisotropic_exchange(J, gL, gR, theta_so, n_so, B):
    """Eq. 17 for fields B ([...][3]): (Jt [...][3][3], |J_perp|, J_par,
    delta E_Z)."""
    B = np.asarray(B, dtype=np.float64)
    Jhat = J * axis_rotation(n_so, -2.0 * theta_so)
    RL = to_z(np.einsum("ij,...j->...i", gL, B))
    RR = to_z(np.einsum("ij,...j->...i", gR, B))
    Jt = RL @ Jhat @ np.swapaxes(RR, -1, -2)
    jperp = 0.5 * np.hypot(Jt[..., 0, 0] + Jt[..., 1, 1], Jt[..., 0, 1] - Jt[..., 1, 0])
    _, db = zeeman_fields(gL, gR, theta_so, n_so, B)
    return Jt, jperp, Jt[..., 2, 2], np.linalg.norm(db, axis=-1)


def field_directions(b_abs, thetas, phis):
    """B = b_abs (sin th cos ph, sin th sin ph, cos th) on the grid
    [len(thetas)][len(phis)][3]."""
    th, ph = np.meshgrid(np.asarray(thetas, dtype=np.float64), np.asarray(phis, dtype=np.float64), indexing="ij")
    return b_abs * np.stack([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)], axis=-1)


def exchange_maps(J, gL, gR, theta_so, n_so, b_abs, thetas, phis):
    """|J_perp|, J_par and delta E_Z over the field directions (Fig. 6 maps)."""
    _, jp, jl, dz = anisotropic_exchange(J, gL, gR, theta_so, n_so, field_directions(b_abs, thetas, phis))
    return jp, jl, dz


def magnetic_spectrum(u_minus_eps, t, gL, gR, theta_so, n_so, B):
    """Eigenvalues [...][5] of Eq. 16 for fields B [...][3]."""
    bbar, db = zeeman_fields(gL, gR, theta_so, n_so, B)
    return np.linalg.eigvalsh(hamiltonian_b(u_minus_eps, t, bbar, db))
