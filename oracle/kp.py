"""Plain FP64 assembly of the discretised 6x6 k.p hole Hamiltonian (CSR).

TEST INFRASTRUCTURE.  Only tests, the smoke check and the CPU-baseline leg
of the benchmark may use this module; the product path never does.

What is assembled (the paper's Eqs. 2b and 5-6a, Sec. II B and III A):
    H_NI = H_LK + H_PB + V,  written in the |X,Y,Z> x {up,down} basis as
    U H_LK U^dag = H_DKK + H_SOI and H'_PB = U H_PB U^dag (Eq. 5), on a
    uniform finite-difference grid with Dirichlet walls (Sec. II B), plus a
    magnetic field through Peierls phases and a Zeeman term.

Conventions where the paper is silent (each is one written reading, shared
with the CUDA path only through this text, never through code):

* hole picture, positive kinetic energy; "lowest" = smallest eigenvalues;
  V is the hole potential energy and enters as +V;
* basis index per point b = 3*s + o, o in (X, Y, Z), s in (up, down);
* H_DKK(k) = C * sum_ab D_ijab k_a k_b (x) 1_spin with C = hbar^2/2m0 and
  D_iiii = g1 + 4 g2, D_iijj = g1 - 2 g2 (i != j),
  D_ijij = D_ijji = 3 g3 (i != j), zero otherwise; rotated into the grid
  frame on all four indices with the rows of `rot`;
* H_SOI = (Delta/3) (1 - L.sigma) with (L_k)_ij = -i eps_kij: 0 on j = 3/2,
  Delta on j = 1/2;
* H'_PB_ij = sum_ab De_ijab eps_ab with the same tensor form,
  l = -(a_v + 2b), m = -(a_v - b), n = -sqrt(3) d  (De_iiii = l,
  De_iijj = m, De_ijij = De_ijji = n/2);
* k = -i grad: second derivative (2 f0 - f+ - f-)/h^2 along one axis,
  mixed derivative -(f++ - f+- - f-+ + f--)/(4 h^2): 19 points;
* Peierls: the block coupling row point r to column point r' is multiplied
  by exp(-i theta), theta = A((r + r')/2) . (r' - r) / Phi0, Phi0 = hbar/e;
  symmetric gauge A = B x (r - r_c)/2 about the box centre, Landau gauge
  A = (0, Bz x - Bx z, -By x);
* Zeeman: mu_B B.(gL L + 2 S), S = sigma/2, gL = 3 kappa - 1, which on the
  j = 3/2 states equals 2 kappa mu_B B.J.
"""
from __future__ import annotations

import itertools

import numpy as np
import scipy.sparse as sp

HBAR2_OVER_2M0 = 0.0380998212   # eV nm^2
MU_B = 5.7883818060e-5          # eV / T
PHI0 = 658.2119569              # hbar / e in T nm^2


def levi_civita() -> np.ndarray:
    e = np.zeros((3, 3, 3))
    for i, j, k in itertools.permutations(range(3)):
        e[i, j, k] = np.linalg.det(np.eye(3)[[i, j, k]])
    return e


def orbital_L():
    """l = 1 angular momentum on the Cartesian orbitals: (L_k)_ij = -i eps_kij."""
    eps = levi_civita()
    return [-1j * eps[k] for k in range(3)]


PAULI = [np.array([[0, 1], [1, 0]], dtype=complex),
         np.array([[0, -1j], [1j, 0]], dtype=complex),
         np.array([[1, 0], [0, -1]], dtype=complex)]


def spin_orbital(spin_op, orb_op) -> np.ndarray:
    """Operator on the 6-dim space with index 3*s + o."""
    return np.kron(spin_op, orb_op)


def luttinger_tensor(g1, g2, g3) -> np.ndarray:
    """D_ijab of H_DKK (units of hbar^2/2m0), crystal frame."""
    D = np.zeros((3, 3, 3, 3))
    for i in range(3):
        D[i, i, i, i] = g1 + 4 * g2
        for j in range(3):
            if i != j:
                D[i, i, j, j] = g1 - 2 * g2
                D[i, j, i, j] = 3 * g3
                D[i, j, j, i] = 3 * g3
    return D


def bir_pikus_tensor(a_v, b, d) -> np.ndarray:
    """De_ijab of H'_PB (eV per unit strain), crystal frame."""
    l_, m_, n_ = -(a_v + 2 * b), -(a_v - b), -np.sqrt(3.0) * d
    D = np.zeros((3, 3, 3, 3))
    for i in range(3):
        D[i, i, i, i] = l_
        for j in range(3):
            if i != j:
                D[i, i, j, j] = m_
                D[i, j, i, j] = n_ / 2
                D[i, j, j, i] = n_ / 2
    return D


def rotate_tensor(D, rot) -> np.ndarray:
    """Grid-frame tensor: D'_abcd = R_ai R_bj R_ck R_dl D_ijkl."""
    R = np.asarray(rot, dtype=np.float64)
    return np.einsum("ai,bj,ck,dl,ijkl->abcd", R, R, R, R, D)


def spin_orbit_matrix(delta) -> np.ndarray:
    L = orbital_L()
    LS = sum(spin_orbital(PAULI[k], L[k]) for k in range(3))
    return (delta / 3.0) * (np.eye(6) - LS)


def zeeman_matrix(B, kappa) -> np.ndarray:
    L = orbital_L()
    gL = 3.0 * kappa - 1.0
    out = np.zeros((6, 6), dtype=complex)
    for k in range(3):
        out += B[k] * (gL * spin_orbital(np.eye(2), L[k]) + 2.0 * spin_orbital(PAULI[k] / 2, np.eye(3)))
    return MU_B * out


def stencil_offsets():
    """The 18 neighbour offsets of the 19-point stencil (6 faces, 12 edges)."""
    offs = []
    for a in range(3):
        for s in (1, -1):
            d = [0, 0, 0]
            d[a] = s
            offs.append(tuple(d))
    for a in range(3):
        for b in range(a + 1, 3):
            for sa in (1, -1):
                for sb in (1, -1):
                    d = [0, 0, 0]
                    d[a], d[b] = sa, sb
                    offs.append(tuple(d))
    return offs


def hop_matrices(Dp, h):
    """Real 3x3 coupling of a point to its neighbour at offset delta, and the
    on-site kinetic 3x3, from the grid-frame tensor (finite differences of
    k_a k_b with k = -i grad)."""
    C = HBAR2_OVER_2M0
    center = np.zeros((3, 3))
    hops = {}
    for a in range(3):
        center += 2.0 * C * Dp[:, :, a, a] / h ** 2
    for d in stencil_offsets():
        nz_axes = [a for a in range(3) if d[a] != 0]
        if len(nz_axes) == 1:
            a = nz_axes[0]
            hops[d] = -C * Dp[:, :, a, a] / h ** 2
        else:
            a, b = nz_axes
            hops[d] = -C * (Dp[:, :, a, b] + Dp[:, :, b, a]) * d[a] * d[b] / (4.0 * h ** 2)
    return center, hops


def vector_potential(gauge, B, nx, ny, nz, h):
    """Return A(x, y, z) in T nm for the chosen gauge."""
    B = np.asarray(B, dtype=np.float64)
    c = np.array([(nx + 1) * h, (ny + 1) * h, (nz + 1) * h]) / 2.0
    if gauge == 0:
        def A(x, y, z):
            rx, ry, rz = x - c[0], y - c[1], z - c[2]
            return (0.5 * (B[1] * rz - B[2] * ry),
                    0.5 * (B[2] * rx - B[0] * rz),
                    0.5 * (B[0] * ry - B[1] * rx))
    elif gauge == 1:
        def A(x, y, z):
            return (np.zeros_like(x), B[2] * x - B[0] * z, -B[1] * x)
    else:
        raise ValueError("gauge must be 0 (symmetric) or 1 (Landau)")
    return A


def onsite_orbital(prob_like):
    """Real 3x3 on-site orbital matrix per point: kinetic centre + V + strain,
    shape [n_points][3][3]."""
    p = prob_like
    mat = p.material
    Dp = rotate_tensor(luttinger_tensor(mat["gamma1"], mat["gamma2"], mat["gamma3"]), p.rot)
    center, _ = hop_matrices(Dp, p.h)
    Np = p.nx * p.ny * p.nz
    out = np.broadcast_to(center, (Np, 3, 3)).copy()
    out += p.V.reshape(Np)[:, None, None] * np.eye(3)[None]
    if p.strain is not None:
        De = rotate_tensor(bir_pikus_tensor(mat["a_v"], mat["b"], mat["d"]), p.rot)
        eps = strain_tensor(p.strain.reshape(6, Np))
        out += np.einsum("ijab,pab->pij", De, eps)
    return out


def strain_tensor(comp):
    """[6][Np] components (xx, yy, zz, yz, xz, xy) -> symmetric [Np][3][3]."""
    Np = comp.shape[1]
    e = np.zeros((Np, 3, 3))
    e[:, 0, 0], e[:, 1, 1], e[:, 2, 2] = comp[0], comp[1], comp[2]
    e[:, 1, 2] = e[:, 2, 1] = comp[3]
    e[:, 0, 2] = e[:, 2, 0] = comp[4]
    e[:, 0, 1] = e[:, 1, 0] = comp[5]
    return e


def assemble(prob, periodic: bool = False) -> sp.csr_matrix:
    """CSR matrix of H (complex128, 6 Np x 6 Np), row index 6 p + b.

    Neighbours outside the box (or excluded by the mask) are dropped:
    Dirichlet walls.  `periodic` wraps neighbours instead (used only by the
    bulk-dispersion checks; requires B = 0)."""
    p = prob
    nx, ny, nz, h = p.nx, p.ny, p.nz, p.h
    Np = nx * ny * nz
    mat = p.material
    Dp = rotate_tensor(luttinger_tensor(mat["gamma1"], mat["gamma2"], mat["gamma3"]), p.rot)
    _, hops = hop_matrices(Dp, h)
    B = np.asarray(p.B, dtype=np.float64)
    if periodic and np.any(B != 0):
        raise ValueError("periodic assembly is only defined for B = 0")
    A = vector_potential(p.gauge, B, nx, ny, nz, h)
    mask = None if p.mask is None else p.mask.reshape(Np).astype(bool)

    iz, iy, ix = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    ix, iy, iz = ix.ravel(), iy.ravel(), iz.ravel()
    pidx = ix + nx * (iy + ny * iz)

    rows, cols, vals = [], [], []

    # on-site block: (centre + V + strain) x 1_spin + H_SOI + H_Z
    orb = onsite_orbital(p)
    const6 = spin_orbit_matrix(mat["delta_so"]) + zeeman_matrix(B, mat["kappa"])
    for b1 in range(6):
        for b2 in range(6):
            s1, o1 = divmod(b1, 3)
            s2, o2 = divmod(b2, 3)
            v = np.full(Np, const6[b1, b2], dtype=complex)
            if s1 == s2:
                v = v + orb[:, o1, o2]
            keep = v != 0
            if mask is not None:
                keep &= mask
            rows.append(6 * pidx[keep] + b1)
            cols.append(6 * pidx[keep] + b2)
            vals.append(v[keep])

    for d, M in hops.items():
        jx, jy, jz = ix + d[0], iy + d[1], iz + d[2]
        if periodic:
            jx, jy, jz = jx % nx, jy % ny, jz % nz
            ok = np.ones(Np, dtype=bool)
        else:
            ok = (jx >= 0) & (jx < nx) & (jy >= 0) & (jy < ny) & (jz >= 0) & (jz < nz)
        src = pidx[ok]
        dst = (jx + nx * (jy + ny * jz))[ok]
        if mask is not None:
            keep = mask[src] & mask[dst]
            src, dst = src[keep], dst[keep]
        # theta = A(midpoint) . (r' - r) / Phi0 on the physical coordinates
        x0, y0, z0 = ((src % nx) + 1.0) * h, (((src // nx) % ny) + 1.0) * h, ((src // (nx * ny)) + 1.0) * h
        x1, y1, z1 = ((dst % nx) + 1.0) * h, (((dst // nx) % ny) + 1.0) * h, ((dst // (nx * ny)) + 1.0) * h
        if np.any(B != 0):
            Ax, Ay, Az = A(0.5 * (x0 + x1), 0.5 * (y0 + y1), 0.5 * (z0 + z1))
            theta = (Ax * (x1 - x0) + Ay * (y1 - y0) + Az * (z1 - z0)) / PHI0
            phase = np.exp(-1j * theta)
        else:
            phase = np.ones(src.shape, dtype=complex)
        for o1 in range(3):
            for o2 in range(3):
                if M[o1, o2] == 0.0:
                    continue
                for s in range(2):
                    rows.append(6 * src + 3 * s + o1)
                    cols.append(6 * dst + 3 * s + o2)
                    vals.append(M[o1, o2] * phase)

    r = np.concatenate(rows)
    c = np.concatenate(cols)
    v = np.concatenate(vals)
    H = sp.csr_matrix((v, (r, c)), shape=(6 * Np, 6 * Np))
    H.sum_duplicates()
    return H


def matvec(H, X):
    """Y = H X for a CSR H and a dense block X [N][m] (row-major)."""
    return np.asarray(H @ X)


def assemble_h0(prob, periodic: bool = False) -> sp.csr_matrix:
    """CSR matrix of the spin-independent single-particle Hamiltonian
    H0 = H_DKK + V + H'_PB (Sec. II C, Eq. 6a), 3 Np x 3 Np, row index 3 p + o
    (o = X, Y, Z).  Without spin-orbit coupling and magnetic field the 6x6
    operator is the identity in spin times H0, so H0 is its spin-up block,
    taken here from the 6x6 assembly with delta_so = 0 and B = 0."""
    if np.any(np.asarray(prob.B, dtype=np.float64) != 0):
        raise ValueError("H0 has no magnetic field: B must be zero")
    mat = dict(prob.material)
    mat["delta_so"] = 0.0
    H6 = assemble(prob.with_(material=mat), periodic=periodic).tocsr()
    Np = prob.nx * prob.ny * prob.nz
    idx = (6 * np.arange(Np)[:, None] + np.arange(3)[None, :]).ravel()
    return H6[idx][:, idx].tocsr()
