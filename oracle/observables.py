"""Plain FP64 hole density and Hellmann-Feynman gradients.

TEST INFRASTRUCTURE.  Only tests, the smoke check and the CPU-baseline leg
of the benchmark may use this module; the product path never does.

* density (Sec. II B: eigenstates -> hole density fed to Poisson):
      rho(r) = sum_i w_i sum_b |psi_i(r, b)|^2   (discrete norm, no h^3)
* Hellmann-Feynman (dE_i/dx = <psi_i| dH/dx |psi_i> for normalised psi_i):
      dL/dV(r)      = sum_i g_i sum_b |psi_i(r, b)|^2        (dH/dV(r) = 1 at r)
      dL/deps_c(r)  = sum_i g_i psi_i(r)^dag (dH'_PB/deps_c x 1_spin) psi_i(r)
      dL/dalpha_g   = sum_r dL/dV(r) Phi_g(r)               (V = V0 + sum alpha_g Phi_g)
  with g_i = dL/dE_i.
"""
from __future__ import annotations

import numpy as np

from .kp import bir_pikus_tensor, rotate_tensor

# strain component c -> tensor indices (a, b): xx, yy, zz, yz, xz, xy
STRAIN_PAIRS = [(0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1)]


def density(evecs, w, bands=6):
    """evecs: [bands Np][n] complex, w: [n] -> rho [Np] (bands = 6, or 3 for
    the spin-independent H0)."""
    N, n = evecs.shape
    P = np.abs(evecs) ** 2                         # [bands Np][n]
    per_state = P.reshape(N // bands, bands, n).sum(axis=1)  # [Np][n]
    return per_state @ np.asarray(w, dtype=np.float64)


def strain_derivative_matrices(material, rot):
    """dH'_PB/deps_c (real 3x3, grid frame) for the six input components."""
    De = rotate_tensor(bir_pikus_tensor(material["a_v"], material["b"], material["d"]), rot)
    out = []
    for a, b in STRAIN_PAIRS:
        if a == b:
            out.append(De[:, :, a, a].copy())
        else:
            out.append(De[:, :, a, b] + De[:, :, b, a])
    return out


def hf_gradients(evecs, g, material, rot, levers=None, bands=6):
    """Returns (dL/dV [Np], dL/deps [6][Np], dL/dalpha [n_gates] or None);
    bands = 3 for the spin-independent H0 (one spin)."""
    N, n = evecs.shape
    Np = N // bands
    g = np.asarray(g, dtype=np.float64)
    dV = density(evecs, g, bands)
    psi = evecs.reshape(Np, bands // 3, 3, n)       # [p][s][o][i]
    dE = np.zeros((6, Np))
    for c, M in enumerate(strain_derivative_matrices(material, rot)):
        # sum_i g_i sum_s psi^dag M psi
        q = np.einsum("psoi,ok,pski->pi", psi.conj(), M, psi).real
        dE[c] = q @ g
    dA = None
    if levers is not None:
        dA = levers.reshape(levers.shape[0], Np) @ dV
    return dV, dE, dA
