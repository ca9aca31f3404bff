"""FP64 oracle of the magnetic two-hole model and the anisotropic exchange
(Sec. III B, Eqs. 16-17).  Test infrastructure only.

Inputs: the symmetric g-tensors g_L, g_R of the two dots, the spin-orbit
axis n_so and angle theta_so, the field B, the tunnel coupling t and the
charging term U - eps.

* Eq. 16, basis {S(0,2), S(1,1), T+(1,1), T-(1,1), T0(1,1)}:
      bbar = mu_B (R(-theta_so) g_L + R(theta_so) g_R) B / 2,
      db   = mu_B (R(-theta_so) g_L - R(theta_so) g_R) B / 2,
  with the 5x5 matrix exactly as printed there.
* t = Delta / sqrt(2) from the bonding/anti-bonding separation Delta;
  J = 2 t^2 / (U - eps), so U - eps = 2 t^2 / J for the J the CI gives.
* Eq. 17: Jhat = J R(-2 theta_so); Jt = R_L Jhat R_R^T;
  |J_perp| = (1/2) sqrt((Jt_xx + Jt_yy)^2 + (Jt_xy - Jt_yx)^2), J_par = Jt_zz.

Readings (the paper leaves them open):
* R(a) is the rotation by the angle a about n_so (right-hand rule); the
  relative rotation of the two dots' spin frames, R(-theta)^T R(theta),
  is then R(2 theta_so), the angle the paper attaches to R;
* R_L is the rotation that carries n_L = g_L B / |g_L B| onto the lab z
  axis along the shortest arc (so that Jt is Jhat in the two qubit frames
  and Jt_zz = n_L . Jhat n_R); any other choice differs by rotations about
  the qubit axes, which leave |J_perp| and J_par unchanged;
* delta E_Z = |db|.
"""
from __future__ import annotations

import numpy as np

from .kp import MU_B


def rotation(axis, angle):
    """Rotation by `angle` about the unit vector `axis` (Rodrigues)."""
    n = np.asarray(axis, dtype=np.float64)
    n = n / np.linalg.norm(n)
    K = np.array([[0.0, -n[2], n[1]], [n[2], 0.0, -n[0]], [-n[1], n[0], 0.0]])
    return np.eye(3) + np.sin(angle) * K + (1.0 - np.cos(angle)) * (K @ K)


def onto_z(n):
    """Shortest-arc rotation R with R n = z for a unit vector n."""
    n = np.asarray(n, dtype=np.float64)
    n = n / np.linalg.norm(n)
    z = np.array([0.0, 0.0, 1.0])
    c = float(n @ z)
    ax = np.cross(n, z)
    s = np.linalg.norm(ax)
    if s < 1e-15:
        return np.eye(3) if c > 0 else rotation([1.0, 0.0, 0.0], np.pi)
    return rotation(ax / s, np.arctan2(s, c))


def zeeman_fields(gL, gR, theta_so, n_so, B):
    """(bbar, db) of Eq. 16, eV."""
    Rm, Rp = rotation(n_so, -theta_so), rotation(n_so, theta_so)
    B = np.asarray(B, dtype=np.float64)
    bbar = MU_B * (Rm @ gL + Rp @ gR) @ B / 2.0
    db = MU_B * (Rm @ gL - Rp @ gR) @ B / 2.0
    return bbar, db


def hamiltonian_b(u_minus_eps, t, bbar, db):
    """The 5x5 matrix of Eq. 16."""
    r2 = np.sqrt(2.0)
    H = np.zeros((5, 5), dtype=complex)
    H[0, 0] = u_minus_eps
    H[0, 1] = H[1, 0] = r2 * t
    H[1, 2] = -(db[0] + 1j * db[1]) / r2
    H[1, 3] = (db[0] - 1j * db[1]) / r2
    H[1, 4] = db[2]
    H[2, 1] = -(db[0] - 1j * db[1]) / r2
    H[2, 2] = bbar[2]
    H[2, 4] = (bbar[0] - 1j * bbar[1]) / r2
    H[3, 1] = (db[0] + 1j * db[1]) / r2
    H[3, 3] = -bbar[2]
    H[3, 4] = (bbar[0] + 1j * bbar[1]) / r2
    H[4, 1] = db[2]
    H[4, 2] = (bbar[0] + 1j * bbar[1]) / r2
    H[4, 3] = (bbar[0] - 1j * bbar[1]) / r2
    return H


def tunnel_coupling(delta):
    return delta / np.sqrt(2.0)


def u_minus_eps(t, J):
    return 2.0 * t * t / J


def anisotropic_exchange(J, gL, gR, theta_so, n_so, B):
    """(Jt, |J_perp|, J_par, delta E_Z) for one field B (Eq. 17)."""
    B = np.asarray(B, dtype=np.float64)
    Jhat = J * rotation(n_so, -2.0 * theta_so)
    nL = gL @ B
    nR = gR @ B
    RL, RR = onto_z(nL / np.linalg.norm(nL)), onto_z(nR / np.linalg.norm(nR))
    Jt = RL @ Jhat @ RR.T
    jperp = 0.5 * np.sqrt((Jt[0, 0] + Jt[1, 1]) ** 2 + (Jt[0, 1] - Jt[1, 0]) ** 2)
    _, db = zeeman_fields(gL, gR, theta_so, n_so, B)
    return Jt, jperp, Jt[2, 2], np.linalg.norm(db)


def exchange_maps(J, gL, gR, theta_so, n_so, b_abs, thetas, phis):
    """|J_perp|, J_par and delta E_Z over polar angles `thetas` and azimuths
    `phis` of a field of magnitude b_abs (arrays [len(thetas)][len(phis)])."""
    jp = np.zeros((len(thetas), len(phis)))
    jl = np.zeros_like(jp)
    dz = np.zeros_like(jp)
    for a, th in enumerate(thetas):
        for b, ph in enumerate(phis):
            B = b_abs * np.array([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)])
            _, jp[a, b], jl[a, b], dz[a, b] = anisotropic_exchange(J, gL, gR, theta_so, n_so, B)
    return jp, jl, dz
