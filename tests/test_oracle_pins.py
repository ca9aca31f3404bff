"""Pins of the FP64 oracle against facts fixed outside the oracle itself.

Each test checks the oracle against a closed form, an independently written
textbook matrix, a physical invariant or brute force, chosen so that a
plausible mistake (a dropped term, a wrong sign or index, a transposed
operand) fails at least one of them.
"""
import numpy as np
import pytest

import inputs
from oracle import eig, kp, observables
from tests.metrics import subspace_sin_angle

C = kp.HBAR2_OVER_2M0


def _box(nx, ny, nz, h=1.0, **kw):
    return inputs.small_problem(nx, ny, nz, h=h, **kw)


# --------------------------------------------------------------------------
# closed form: gamma2 = gamma3 = 0, V = 0, B = 0, no strain -> particle in a
# box, E_k x4 (j = 3/2) and E_k + Delta x2 (j = 1/2), any Delta
@pytest.mark.parametrize("shape,h,delta", [((5, 4, 3), 0.7, 0.044), ((6, 3, 4), 0.5, 0.3)])
def test_box_closed_form(shape, h, delta):
    p = _box(*shape, h=h, strain=False, noise_mev=0.0)
    p.material.update(gamma2=0.0, gamma3=0.0, delta_so=delta)
    p.V[:] = 0.0
    w = eig.all_eigenvalues_dense(kp.assemble(p))
    g1 = p.material["gamma1"]
    ref = []
    nx, ny, nz = shape
    for kx in range(1, nx + 1):
        for ky in range(1, ny + 1):
            for kz in range(1, nz + 1):
                E = C * g1 * sum(2 - 2 * np.cos(k * np.pi / (n + 1))
                                 for k, n in ((kx, nx), (ky, ny), (kz, nz))) / h ** 2
                ref += [E] * 4 + [E + delta] * 2
    assert np.abs(w - np.sort(ref)).max() < 1e-12


# --------------------------------------------------------------------------
# textbook 6x6 Luttinger-Kohn matrix in the |J, m_j> basis (P, Q, R, S form),
# typed independently of the oracle's tensor construction
def _pqrs_kinetic(K, g1, g2, g3):
    """Luttinger P, Q, R, S with k_i k_j -> K[i, j] (crystal frame)."""
    kx2, ky2, kz2 = K[0, 0], K[1, 1], K[2, 2]
    P = C * g1 * (kx2 + ky2 + kz2)
    Q = C * g2 * (kx2 + ky2 - 2 * kz2)
    R = C * np.sqrt(3) * (-g2 * (kx2 - ky2) + 2j * g3 * K[0, 1])
    S = C * 2 * np.sqrt(3) * g3 * (K[0, 2] - 1j * K[1, 2])
    return P, Q, R, S


def _pqrs_strain(e, a_v, b, d):
    """Bir-Pikus P, Q, R, S for the strain tensor e (crystal frame)."""
    P = -a_v * (e[0, 0] + e[1, 1] + e[2, 2])
    Q = -0.5 * b * (e[0, 0] + e[1, 1] - 2 * e[2, 2])
    R = 0.5 * np.sqrt(3) * b * (e[0, 0] - e[1, 1]) - 1j * d * e[0, 1]
    S = -d * (e[0, 2] - 1j * e[1, 2])
    return P, Q, R, S


def _lk_textbook(P, Q, R, S, delta):
    s2, s32, cj = np.sqrt(2), np.sqrt(1.5), np.conj
    return np.array([
        [P + Q, -S, R, 0, -S / s2, s2 * R],
        [-cj(S), P - Q, 0, R, -s2 * Q, s32 * S],
        [cj(R), 0, P - Q, S, s32 * cj(S), s2 * Q],
        [0, cj(R), cj(S), P + Q, -s2 * cj(R), -cj(S) / s2],
        [-cj(S) / s2, -s2 * Q, s32 * S, -s2 * R, P + delta, 0],
        [s2 * cj(R), s32 * cj(S), s2 * Q, -S / s2, 0, P + delta]], dtype=complex)


def _plane_wave_symbol(H, p, kvec):
    """6x6 symbol of a periodic, translation-invariant H at wave vector k,
    read off by applying H to the six plane waves exp(i k.r) e_b."""
    nx, ny, nz, h = p.nx, p.ny, p.nz, p.h
    iz, iy, ix = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    ph = np.exp(1j * h * (kvec[0] * ix + kvec[1] * iy + kvec[2] * iz)).ravel()
    Np = nx * ny * nz
    X = np.zeros((6 * Np, 6), dtype=complex)
    for b in range(6):
        X[b::6, b] = ph
    Y = H @ X
    return Y[0:6, :] / ph[0]


@pytest.mark.parametrize("rot", ["identity", "device"])
def test_bulk_symbol_matches_textbook_luttinger_kohn(rot):
    """Periodic CSR symbol == textbook LK matrix with k_a k_b replaced by the
    finite-difference symbols (2-2cos)/h^2 and sin sin/h^2 in the grid frame,
    transformed to the crystal frame with the rotation."""
    p = _box(6, 6, 6, h=0.5, strain=False, noise_mev=0.0, rot=rot)
    p.V[:] = 0.0
    H = kp.assemble(p, periodic=True)
    m = p.material
    R = p.rot
    for j in [(1, 0, 0), (0, 0, 2), (1, 1, 1), (1, 2, 3), (2, -1, 1), (3, 3, 0)]:
        k = 2 * np.pi * np.array(j) / (6 * p.h)
        Ks = np.empty((3, 3))
        for a in range(3):
            for b in range(3):
                Ks[a, b] = ((2 - 2 * np.cos(k[a] * p.h)) if a == b
                            else np.sin(k[a] * p.h) * np.sin(k[b] * p.h)) / p.h ** 2
        Kc = R.T @ Ks @ R
        sym = _plane_wave_symbol(H, p, k)
        assert np.abs(sym - sym.conj().T).max() < 1e-13
        e_or = np.linalg.eigvalsh(sym)
        e_tb = np.linalg.eigvalsh(_lk_textbook(*_pqrs_kinetic(Kc, m["gamma1"], m["gamma2"], m["gamma3"]),
                                               m["delta_so"]))
        assert np.abs(e_or - e_tb).max() < 1e-12


def test_luttinger_dispersion_001_111():
    """Delta -> infinity (projection on j = 3/2): along [001] the heavy/light
    holes are C(g1 -+ 2 g2) k^2 and along [111] C(g1 -+ 2 g3) k^2 (with the
    finite-difference symbols of k_a k_b)."""
    p = _box(6, 6, 6, h=0.5, strain=False, noise_mev=0.0)
    p.V[:] = 0.0
    m = p.material
    H = kp.assemble(p, periodic=True)
    so = kp.spin_orbit_matrix(1.0)
    w, U = np.linalg.eigh(so)
    P32 = U[:, np.abs(w) < 1e-12]                 # j = 3/2 eigenspace, 4 dims
    assert P32.shape[1] == 4
    h = p.h
    for j in (1, 2):
        k = 2 * np.pi * j / (6 * h)
        Kd = (2 - 2 * np.cos(k * h)) / h ** 2
        S = np.sin(k * h) ** 2 / h ** 2
        e = np.linalg.eigvalsh(P32.conj().T @ _plane_wave_symbol(H, p, np.array([0, 0, k])) @ P32)
        assert np.allclose(e, np.sort([C * (m["gamma1"] - 2 * m["gamma2"]) * Kd] * 2
                                      + [C * (m["gamma1"] + 2 * m["gamma2"]) * Kd] * 2), atol=1e-12)
        e = np.linalg.eigvalsh(P32.conj().T @ _plane_wave_symbol(H, p, np.array([k, k, k])) @ P32)
        hh = C * (3 * m["gamma1"] * Kd - 6 * m["gamma3"] * S)
        lh = C * (3 * m["gamma1"] * Kd + 6 * m["gamma3"] * S)
        assert np.allclose(e, np.sort([hh, hh, lh, lh]), atol=1e-12)


# --------------------------------------------------------------------------
def test_spin_orbit_spectrum():
    w = np.linalg.eigvalsh(kp.spin_orbit_matrix(0.044))
    assert np.allclose(w, [0, 0, 0, 0, 0.044, 0.044], atol=1e-15)


def test_zeeman_on_j32_is_isotropic_luttinger_term():
    """On the j = 3/2 states the Zeeman term equals 2 kappa mu_B B.J:
    eigenvalues +-3 kappa mu_B |B| and +-kappa mu_B |B|; zero on j = 1/2 x j = 3/2
    is not required, only the projected spectrum."""
    kappa = -0.42
    rng = np.random.default_rng(3)
    w, U = np.linalg.eigh(kp.spin_orbit_matrix(1.0))
    P32 = U[:, np.abs(w) < 1e-12]
    for _ in range(3):
        B = rng.standard_normal(3)
        Z = P32.conj().T @ kp.zeeman_matrix(B, kappa) @ P32
        e = np.linalg.eigvalsh(Z)
        b = kp.MU_B * np.linalg.norm(B) * abs(kappa)
        assert np.allclose(e, [-3 * b, -b, b, 3 * b], atol=1e-18)


# --------------------------------------------------------------------------
@pytest.mark.parametrize("rot,bound", [("identity", 0.0), ("device", 1e-16)])
def test_hermitian(rot, bound):
    """Exactly Hermitian in the crystal frame; to rounding of the rotated
    tensor (relative to the largest entry) in the device frame."""
    p = _box(5, 4, 3, rot=rot, B=(0.7, -0.4, 1.1))
    H = kp.assemble(p)
    D = (H - H.conj().T).tocoo()
    worst = np.abs(D.data).max() if D.nnz else 0.0
    assert worst <= bound * abs(H).max()


def test_kramers_doubling_at_zero_field():
    p = _box(5, 4, 4, rot="device", strain=True)
    w = eig.all_eigenvalues_dense(kp.assemble(p))
    assert np.abs(w[0::2] - w[1::2]).max() < 1e-12
    assert np.min(w[2::2] - w[1:-1:2]) > 1e-9      # doublets, not quartets everywhere


def test_gauge_invariance():
    B = (0.9, -1.3, 2.0)
    p0 = _box(5, 4, 4, rot="device", B=B, gauge=0)
    p1 = p0.with_(gauge=1)
    w0 = eig.all_eigenvalues_dense(kp.assemble(p0))
    w1 = eig.all_eigenvalues_dense(kp.assemble(p1))
    assert np.abs(w0 - w1).max() < 1e-12
    # and the field does something
    w00 = eig.all_eigenvalues_dense(kp.assemble(p0.with_(B=np.zeros(3))))
    assert np.abs(w0 - w00).max() > 1e-5


def test_time_reversal_B_minus_B():
    p = _box(4, 4, 3, rot="device", B=(0.3, 0.8, -0.5))
    w0 = eig.all_eigenvalues_dense(kp.assemble(p))
    w1 = eig.all_eigenvalues_dense(kp.assemble(p.with_(B=-p.B)))
    assert np.abs(w0 - w1).max() < 1e-12


@pytest.mark.parametrize("gauge", [0, 1])
def test_plaquette_flux(gauge):
    """Product of link phases around an elementary plaquette is
    exp(-i B.n h^2 / Phi0) (Stokes), for all three plaquette orientations."""
    B = np.array([3.0, -2.0, 5.0])
    p = _box(4, 4, 4, h=0.8, strain=False, noise_mev=0.0, B=B, gauge=gauge)
    p.material.update(gamma2=0.0, gamma3=0.0)   # face hops diagonal, edges zero
    H = kp.assemble(p).tolil()
    nx, ny = p.nx, p.ny

    def idx(x, y, z):
        return 6 * (x + nx * (y + ny * z))

    for a, b in [(0, 1), (1, 2), (2, 0)]:
        r0 = np.array([1, 1, 1])
        ea, eb = np.eye(3, dtype=int)[a], np.eye(3, dtype=int)[b]
        loop = [r0, r0 + ea, r0 + ea + eb, r0 + eb, r0]
        prod = 1.0 + 0j
        for u, v in zip(loop[:-1], loop[1:]):
            prod *= H[idx(*u), idx(*v)]
        n = np.cross(ea, eb)
        flux = B @ n * p.h ** 2
        ref = np.exp(-1j * flux / kp.PHI0)
        assert abs(prod / abs(prod) - ref) < 1e-13


def test_hydrostatic_strain_rigid_shift():
    e = 3e-4
    p = _box(4, 4, 3, rot="device", strain=False)
    w0 = eig.all_eigenvalues_dense(kp.assemble(p))
    eps = np.zeros((6, p.nz, p.ny, p.nx))
    eps[0:3] = e
    w1 = eig.all_eigenvalues_dense(kp.assemble(p.with_(strain=eps)))
    assert np.abs(w1 - w0 - (-3 * p.material["a_v"] * e)).max() < 1e-13


def test_isotropic_tensor_rotation_invariant():
    p = _box(4, 3, 3, strain=False)
    p.material.update(gamma3=p.material["gamma2"])
    H0 = kp.assemble(p)
    H1 = kp.assemble(p.with_(rot=inputs.ROT_DEVICE.copy()))
    assert abs(H0 - H1).max() < 1e-13


@pytest.mark.parametrize("rot", ["identity", "device"])
def test_strain_and_kinetic_match_textbook_bir_pikus(rot):
    """Bulk symbol with a uniform random strain (grid frame) == textbook
    LK + Bir-Pikus matrix (P_e = -a_v tr e, Q_e = -b/2 (exx + eyy - 2 ezz),
    R_e = sqrt3/2 b (exx - eyy) - i d exy, S_e = -d (exz - i eyz)) in the
    crystal frame, at k = 0 and at finite k."""
    p = _box(6, 6, 6, h=0.5, strain=False, noise_mev=0.0, rot=rot)
    p.V[:] = 0.0
    m = p.material
    R = p.rot
    rng = np.random.default_rng(21)
    eg = rng.uniform(-2e-3, 2e-3, size=(3, 3))
    eg = 0.5 * (eg + eg.T)
    comp = [eg[0, 0], eg[1, 1], eg[2, 2], eg[1, 2], eg[0, 2], eg[0, 1]]
    eps = np.zeros((6, 6, 6, 6))
    for c in range(6):
        eps[c] = comp[c]
    H = kp.assemble(p.with_(strain=eps), periodic=True)
    ec = R.T @ eg @ R
    for j in [(0, 0, 0), (1, 2, 3), (2, 0, -1)]:
        k = 2 * np.pi * np.array(j) / (6 * p.h)
        Ks = np.empty((3, 3))
        for a in range(3):
            for b in range(3):
                Ks[a, b] = ((2 - 2 * np.cos(k[a] * p.h)) if a == b
                            else np.sin(k[a] * p.h) * np.sin(k[b] * p.h)) / p.h ** 2
        Pk, Qk, Rk, Sk = _pqrs_kinetic(R.T @ Ks @ R, m["gamma1"], m["gamma2"], m["gamma3"])
        Pe, Qe, Re, Se = _pqrs_strain(ec, m["a_v"], m["b"], m["d"])
        ref = np.linalg.eigvalsh(_lk_textbook(Pk + Pe, Qk + Qe, Rk + Re, Sk + Se, m["delta_so"]))
        got = np.linalg.eigvalsh(_plane_wave_symbol(H, p, k))
        assert np.abs(got - ref).max() < 1e-12


# --------------------------------------------------------------------------
def test_mask_equals_smaller_box():
    """Masking the outer layer of a box gives exactly the spectrum of the
    inner box (Dirichlet walls), with the same point-wise potential."""
    big = _box(7, 6, 5, strain=False, noise_mev=0.0)
    inner = _box(5, 4, 3, strain=False, noise_mev=0.0)
    rng = np.random.default_rng(5)
    Vin = rng.uniform(-0.01, 0.01, size=(3, 4, 5))
    Vbig = np.zeros((5, 6, 7))
    Vbig[1:-1, 1:-1, 1:-1] = Vin
    mask = np.zeros((5, 6, 7), dtype=np.uint8)
    mask[1:-1, 1:-1, 1:-1] = 1
    wb = eig.all_eigenvalues_dense(kp.assemble(big.with_(V=Vbig, mask=mask)), mask=mask)
    wi = eig.all_eigenvalues_dense(kp.assemble(inner.with_(V=Vin)))
    assert np.abs(wb - wi).max() < 1e-12


# --------------------------------------------------------------------------
def test_block_lanczos_matches_dense():
    for p in (inputs.config1(), _box(6, 6, 6, rot="device", B=(0.4, 0.2, -0.9))):
        H = kp.assemble(p)
        wd, vd = eig.lowest_dense(H, 12)
        wl, vl, res, _ = eig.lowest_block_lanczos(H, 8, return_residuals=True)
        assert np.abs(wl - wd[:8]).max() < 1e-12
        assert res.max() < 1e-11
        # same invariant subspace (clusters are not cut at 8 for these cases)
        assert subspace_sin_angle(vd[:, :8], vl) < 1e-9


def test_arpack_matches_dense_and_block_lanczos():
    """The ARPACK path (used for the largest grids at B != 0) against dense
    LAPACK on config 1 with a field and against block Lanczos on a 6x6x6
    device-frame grid with strain and a tilted field."""
    c1 = inputs.config1().with_(B=np.array([0.0, 0.3, 0.6]))
    for p, ref in ((c1, "dense"), (_box(6, 6, 6, rot="device", B=(0.4, 0.2, -0.9)), "lanczos")):
        H = kp.assemble(p)
        if ref == "dense":
            wr, vr = eig.lowest_dense(H, 12)
        else:
            wr, vr = eig.lowest_block_lanczos(H, 12, tol=1e-12)
        wa, va, res, nmv = eig.lowest_arpack(H, 10, return_residuals=True)
        assert np.abs(wa - wr[:10]).max() < 1e-12
        assert res.max() < 1e-11
        assert np.all(np.diff(wr[:11]) > 1e-9)      # no exact degeneracy at B != 0
        assert subspace_sin_angle(vr[:, :10], va) < 1e-9


def test_dense_matches_numpy_full_diagonalisation():
    p = _box(4, 3, 3, rot="device", B=(0.0, 0.5, 0.5))
    H = kp.assemble(p)
    w, v = eig.lowest_dense(H, 6)
    wn = np.linalg.eigvalsh(H.toarray())
    assert np.abs(w - wn[:6]).max() < 1e-13
    r = H @ v - v * w
    assert np.abs(r).max() < 1e-12


# --------------------------------------------------------------------------
def test_density_normalisation_and_pointwise():
    p = _box(4, 3, 3)
    H = kp.assemble(p)
    w, v = eig.lowest_dense(H, 6)
    wt = np.array([1.0, 0.5, 2.0, -1.0, 0.25, 3.0])
    rho = observables.density(v, wt)
    assert abs(rho.sum() - wt.sum()) < 1e-12
    # brute-force pointwise loop
    Np = p.n_points
    ref = np.zeros(Np)
    for i in range(6):
        for pt in range(Np):
            for b in range(6):
                ref[pt] += wt[i] * abs(v[6 * pt + b, i]) ** 2
    assert np.abs(rho - ref).max() < 1e-14


def _doublet_loss_weights(n):
    """Loss = (mean of doublet 1 - mean of doublet 0) + sum_{i<n} E_i as dL/dE."""
    g = np.ones(n)
    g[0:2] += -0.5
    g[2:4] += 0.5
    return g


def test_hellmann_feynman_vs_finite_differences():
    """dL/dV, dL/deps and dL/dalpha from HF equal central differences of the
    dense eigenvalues (B = 0: doublet-averaged loss, well defined)."""
    p = _box(5, 4, 3, rot="device", strain=True, levers=3)
    n = 8
    g = _doublet_loss_weights(n)

    def loss(q):
        w, _ = eig.lowest_dense(kp.assemble(q), n)
        return g @ w

    w, v = eig.lowest_dense(kp.assemble(p), n)
    dV, dEps, dA = observables.hf_gradients(v, g, p.material, p.rot, p.levers)
    rng = np.random.default_rng(11)
    d = 1e-5
    for _ in range(2):
        u = rng.standard_normal(p.V.shape)
        fd = (loss(p.with_(V=p.V + d * u)) - loss(p.with_(V=p.V - d * u))) / (2 * d)
        assert abs(fd - dV @ u.ravel()) < 1e-8 * max(1.0, abs(fd))
    for c in (0, 3, 5):
        u = np.zeros_like(p.strain)
        u[c] = rng.standard_normal(p.V.shape)
        de = 1e-6
        fd = (loss(p.with_(strain=p.strain + de * u)) - loss(p.with_(strain=p.strain - de * u))) / (2 * de)
        assert abs(fd - (dEps * u.reshape(6, -1)).sum()) < 1e-6 * max(1.0, abs(fd))
    for gi in range(3):
        fd = (loss(p.with_(V=p.V + d * p.levers[gi])) - loss(p.with_(V=p.V - d * p.levers[gi]))) / (2 * d)
        assert abs(fd - dA[gi]) < 1e-8 * max(1.0, abs(fd))


# --------------------------------------------------------------------------
# the spin-independent H0 (Sec. II C, Eq. 6a): one 3x3-orbital block
@pytest.mark.parametrize("shape,h", [((5, 4, 3), 0.7), ((6, 3, 4), 0.5)])
def test_h0_box_closed_form(shape, h):
    """gamma2 = gamma3 = 0, V = 0, no strain: the three orbitals decouple and
    each is the particle in a box, so every box level appears three times."""
    p = _box(*shape, h=h, strain=False, noise_mev=0.0)
    p.material.update(gamma2=0.0, gamma3=0.0)
    p.V[:] = 0.0
    w = eig.all_eigenvalues_dense(kp.assemble_h0(p))
    g1 = p.material["gamma1"]
    nx, ny, nz = shape
    ref = []
    for kx in range(1, nx + 1):
        for ky in range(1, ny + 1):
            for kz in range(1, nz + 1):
                E = C * g1 * sum(2 - 2 * np.cos(k * np.pi / (n + 1))
                                 for k, n in ((kx, nx), (ky, ny), (kz, nz))) / h ** 2
                ref += [E] * 3
    assert np.abs(w - np.sort(ref)).max() < 1e-12


def _dkk_textbook(K, g1, g2, g3):
    """Dresselhaus-Kittel-Kip 3x3 (hole picture, crystal frame) with
    L = g1 + 4 g2, M = g1 - 2 g2, N = 6 g3 and k_a k_b -> K[a, b]."""
    L, M, N = g1 + 4 * g2, g1 - 2 * g2, 6 * g3
    D = np.empty((3, 3))
    for i in range(3):
        D[i, i] = L * K[i, i] + M * (np.trace(K) - K[i, i])
        for j in range(3):
            if j != i:
                D[i, j] = N * K[i, j]
    return C * D


@pytest.mark.parametrize("rot", ["identity", "device"])
def test_h0_bulk_symbol_matches_textbook_dkk(rot):
    """Periodic H0 applied to the three plane waves exp(i k.r) e_o gives the
    textbook DKK matrix with the finite-difference symbols of k_a k_b."""
    p = _box(6, 6, 6, h=0.5, strain=False, noise_mev=0.0, rot=rot)
    p.V[:] = 0.0
    H = kp.assemble_h0(p, periodic=True)
    m, R = p.material, p.rot
    iz, iy, ix = np.meshgrid(np.arange(6), np.arange(6), np.arange(6), indexing="ij")
    for j in [(1, 0, 0), (1, 1, 1), (1, 2, 3), (2, -1, 1)]:
        k = 2 * np.pi * np.array(j) / (6 * p.h)
        ph = np.exp(1j * p.h * (k[0] * ix + k[1] * iy + k[2] * iz)).ravel()
        X = np.zeros((3 * ph.size, 3), dtype=complex)
        for o in range(3):
            X[o::3, o] = ph
        sym = (H @ X)[0:3, :] / ph[0]
        Ks = np.empty((3, 3))
        for a in range(3):
            for b in range(3):
                Ks[a, b] = ((2 - 2 * np.cos(k[a] * p.h)) if a == b
                            else np.sin(k[a] * p.h) * np.sin(k[b] * p.h)) / p.h ** 2
        Kc = R.T @ Ks @ R
        e_or = np.linalg.eigvalsh(sym)
        e_tb = np.linalg.eigvalsh(_dkk_textbook(Kc, m["gamma1"], m["gamma2"], m["gamma3"]))
        assert np.abs(e_or - e_tb).max() < 1e-12


def test_h0_is_the_spin_block_of_the_full_operator():
    """delta_so = 0, B = 0: the 6x6 operator is 1_spin x H0 (both spin blocks
    equal H0, no spin mixing) and H0 is real symmetric; a field is refused."""
    p = _box(5, 4, 6, h=0.5, strain=True, rot="device")
    p.material.update(delta_so=0.0)
    H6 = kp.assemble(p).tocsr()
    H0 = kp.assemble_h0(p)
    Np = p.nx * p.ny * p.nz
    up = (6 * np.arange(Np)[:, None] + np.arange(3)[None, :]).ravel()
    dn = up + 3
    assert abs(H6[up][:, up] - H0).max() == 0
    assert abs(H6[dn][:, dn] - H0).max() == 0
    assert abs(H6[up][:, dn]).max() == 0
    assert abs(H0.imag).max() == 0 and abs(H0 - H0.T).max() < 1e-15 * abs(H0).max()
    with pytest.raises(ValueError):
        kp.assemble_h0(p.with_(B=(0.0, 0.0, 0.1)))


def test_h0_hellmann_feynman_vs_finite_differences():
    """H0 (3 bands): dL/dV, dL/deps and dL/dalpha from the one-spin HF
    formulas equal central differences of the dense H0 eigenvalues for
    L = (E1 - E0) + sum_{i<6} E_i (H0 levels are not spin-degenerate)."""
    p = _box(5, 4, 3, rot="device", strain=True, levers=2)
    n = 6
    g = np.ones(n)
    g[0] -= 1.0
    g[1] += 1.0

    def loss(q):
        w, _ = eig.lowest_dense(kp.assemble_h0(q), n)
        return g @ w

    w, v = eig.lowest_dense(kp.assemble_h0(p), n)
    assert np.min(np.diff(w)) > 1e-6
    dV, dEps, dA = observables.hf_gradients(v, g, p.material, p.rot, p.levers, bands=3)
    rng = np.random.default_rng(12)
    # close but non-degenerate levels: a step of 1e-6 keeps the O(d^2)
    # truncation of the central difference below 1e-9
    d = 1e-6
    for _ in range(2):
        u = rng.standard_normal(p.V.shape)
        fd = (loss(p.with_(V=p.V + d * u)) - loss(p.with_(V=p.V - d * u))) / (2 * d)
        assert abs(fd - dV @ u.ravel()) < 1e-8 * max(1.0, abs(fd))
    for c in (0, 3, 5):
        u = np.zeros_like(p.strain)
        u[c] = rng.standard_normal(p.V.shape)
        de = 1e-6
        fd = (loss(p.with_(strain=p.strain + de * u)) - loss(p.with_(strain=p.strain - de * u))) / (2 * de)
        assert abs(fd - (dEps * u.reshape(6, -1)).sum()) < 1e-6 * max(1.0, abs(fd))
    for gi in range(2):
        fd = (loss(p.with_(V=p.V + d * p.levers[gi])) - loss(p.with_(V=p.V - d * p.levers[gi]))) / (2 * d)
        assert abs(fd - dA[gi]) < 1e-8 * max(1.0, abs(fd))


# --------------------------------------------------------------------------
# Poisson step of the Schroedinger-Poisson loop (Sec. II B)
from oracle import poisson as poisson_oracle  # noqa: E402


def _end_gates(nx, ny, nz):
    g = np.zeros((nz, ny, nx), dtype=np.uint8)
    g[:, :, 0] = 1
    g[:, :, -1] = 1
    return g


def test_poisson_linear_between_two_gates():
    """No charge, gates at the two x faces (0 and U), zero flux elsewhere:
    the discrete solution is exactly linear in x."""
    nx, ny, nz, h, U = 9, 4, 5, 0.5, 0.7
    g = _end_gates(nx, ny, nz)
    phi_g = np.zeros((nz, ny, nx))
    phi_g[:, :, -1] = U
    phi = poisson_oracle.solve(nx, ny, nz, h, g, phi_g, np.zeros(nx * ny * nz)).reshape(nz, ny, nx)
    ref = U * np.arange(nx) / (nx - 1)
    assert np.abs(phi - ref[None, None, :]).max() < 1e-13


def test_poisson_uniform_charge_quadratic():
    """Uniform hole density c between grounded x faces: -phi'' = (e/eps) c,
    whose discrete solution is the exact quadratic (e/eps) c h^2 i (n-1-i)/2."""
    nx, ny, nz, h, c = 11, 3, 4, 0.5, 2e-3
    g = _end_gates(nx, ny, nz)
    phi = poisson_oracle.solve(nx, ny, nz, h, g, np.zeros((nz, ny, nx)), np.full(nx * ny * nz, c))
    i = np.arange(nx)
    ref = poisson_oracle.e_over_eps() * c * h ** 2 * i * (nx - 1 - i) / 2
    assert np.abs(phi.reshape(nz, ny, nx) - ref[None, None, :]).max() < 1e-12 * ref.max()


def test_poisson_reciprocity():
    """Grounded gates: the potential at b of a unit charge at a equals the
    potential at a of a unit charge at b (symmetric operator)."""
    nx, ny, nz, h = 6, 5, 4, 0.5
    rng = np.random.default_rng(3)
    g = (rng.random((nz, ny, nx)) < 0.15).astype(np.uint8)
    g[0, 0, 0] = 1
    free = np.flatnonzero(g.reshape(-1) == 0)
    a, b = free[3], free[-5]
    ra = np.zeros(nx * ny * nz)
    ra[a] = 1.0
    rb = np.zeros(nx * ny * nz)
    rb[b] = 1.0
    z = np.zeros((nz, ny, nx))
    pa = poisson_oracle.solve(nx, ny, nz, h, g, z, ra)
    pb = poisson_oracle.solve(nx, ny, nz, h, g, z, rb)
    assert abs(pa[b] - pb[a]) < 1e-12 * abs(pa[b])
    assert pa[a] > pa[b] > 0


def test_fermi_level_counts_holes():
    E = np.array([0.010, 0.010, 0.012, 0.012, 0.020, 0.021])
    for kT, n in ((1e-4, 2.0), (1e-3, 3.0), (5e-3, 1.5)):
        mu = poisson_oracle.fermi_level(E, n, kT)
        assert abs(poisson_oracle.occupations(E, mu, kT).sum() - n) < 1e-12


# --------------------------------------------------------------------------
# configuration interaction (Sec. II C, Eqs. 7-15)
from oracle import ci as ci_oracle  # noqa: E402


def _random_integrals(n, rng):
    """Hermitian one-body matrix on 2n spin-orbitals and a spatial two-body
    tensor with the symmetries of a Coulomb operator (built from random
    complex overlap densities and a symmetric positive kernel)."""
    A = rng.standard_normal((2 * n, 2 * n)) + 1j * rng.standard_normal((2 * n, 2 * n))
    h = A + A.conj().T
    npnt = 7
    phi = rng.standard_normal((npnt, n)) + 1j * rng.standard_normal((npnt, n))
    rho = np.einsum("pi,pk->pik", phi.conj(), phi)
    B = rng.standard_normal((npnt, npnt))
    G = B @ B.T + npnt * np.eye(npnt)
    J = np.einsum("pik,pq,qjl->ijkl", rho, G, rho)
    return h, J


@pytest.mark.parametrize("n", [2, 3])
def test_ci_slater_condon_matches_brute_force(n):
    """The determinant-basis CI matrix equals the full two-particle
    Hamiltonian h1 + h2 + C projected on antisymmetric product states."""
    rng = np.random.default_rng(n)
    h, J = _random_integrals(n, rng)
    H, dets = ci_oracle.ci_matrix(h, J, n)
    M = 2 * n
    I = np.eye(M)
    H2 = np.kron(h, I) + np.kron(I, h)
    for a in range(M):
        for b in range(M):
            for c in range(M):
                for d in range(M):
                    if a % 2 == c % 2 and b % 2 == d % 2:
                        H2[a * M + b, c * M + d] += J[a // 2, b // 2, c // 2, d // 2]
    P = np.zeros((M * M, len(dets)))
    for x, (a, b) in enumerate(dets):
        P[a * M + b, x] = 1 / np.sqrt(2)
        P[b * M + a, x] = -1 / np.sqrt(2)
    assert np.abs(P.T @ H2 @ P - H).max() < 1e-12 * np.abs(H).max()
    assert np.abs(H - H.conj().T).max() < 1e-12 * np.abs(H).max()


@pytest.mark.parametrize("n", [2, 3, 4])
def test_ci_spin_labels_without_spin_orbit(n):
    """Without spin-orbit coupling S^2 commutes with H: its eigenvalues are
    exactly 0 (n(n+1)/2 singlets) and 2 (3 n(n-1)/2 triplet states)."""
    s2 = np.linalg.eigvalsh(ci_oracle.spin_squared(n))
    assert np.sum(np.abs(s2) < 1e-12) == n * (n + 1) // 2
    assert np.sum(np.abs(s2 - 2) < 1e-12) == 3 * n * (n - 1) // 2


def test_ci_coulomb_tensor_symmetries_and_exchange_sign():
    """Coulomb integrals of H0 orbitals through the Poisson step: particle
    swap J[ijkl] = J[jilk], Hermiticity J[ijkl] = conj(J[klij]); without
    spin-orbit coupling the two-hole ground state of a double well is a
    singlet (J_ex > 0)."""
    p = inputs.small_problem(12, 6, 6, h=0.5, seed=5, strain=False)
    p.material.update(delta_so=0.0)
    gate = np.zeros((p.nz, p.ny, p.nx), dtype=np.uint8)
    gate[:, :, 0] = 1
    gate[:, :, -1] = 1
    E, phi = ci_oracle.h0_orbitals(p, 2)
    J = ci_oracle.coulomb_tensor(phi, p.nx, p.ny, p.nz, p.h, gate)
    scale = np.abs(J).max()
    assert np.abs(J - J.transpose(1, 0, 3, 2)).max() < 1e-12 * scale
    assert np.abs(J - J.transpose(2, 3, 0, 1).conj()).max() < 1e-12 * scale
    w, s2, jex = ci_oracle.exchange(ci_oracle.ci_matrix(ci_oracle.one_body(E, ci_oracle.orbital_overlaps(phi), 0.0),
                                                        J, 2)[0], 2)
    assert s2[0] < 1e-9 and jex > 0


def _spin_orbitals(phi):
    """Columns 2 i + s: orbital i (three components per point) times spin s,
    embedded in the 6-band row order 6 p + 3 s + o."""
    N3, n = phi.shape
    Np = N3 // 3
    P = phi.reshape(Np, 3, n)
    out = np.zeros((Np, 2, 3, n, 2), dtype=complex)
    for s in range(2):
        out[:, s, :, :, s] = P
    return out.reshape(6 * Np, 2 * n)


@pytest.mark.parametrize("n_orb", [None, 5])
def test_ci_one_body_is_the_projected_full_operator(n_orb):
    """The CI one-body block (H0 energies plus the spin-orbit term between
    H0 orbitals, Eqs. 11-12) equals the full 6x6 operator at B = 0 (pinned
    separately above) projected on the spin-orbitals, entry by entry, since
    H = H0 x 1_spin + H_SOI.  In the complete basis of all 3 Np H0 orbitals
    its spectrum is the full operator's.  The orbitals carry random phases,
    so a dropped conjugate, a transposed overlap O[i,o,j,q] or swapped spin
    indices of the spin-orbit matrix change the entries."""
    p = inputs.small_problem(3, 2, 2, h=0.5, seed=9, rot="device", strain=True)
    nb = 3 * p.n_points
    n = nb if n_orb is None else n_orb
    E, phi = eig.lowest_dense(kp.assemble_h0(p), n)
    rng = np.random.default_rng(17)
    phi = phi * np.exp(2j * np.pi * rng.uniform(size=n))[None, :]
    h1 = ci_oracle.one_body(E, ci_oracle.orbital_overlaps(phi), p.material["delta_so"])
    H = kp.assemble(p).toarray()
    S = _spin_orbitals(phi)
    proj = S.conj().T @ H @ S
    scale = np.abs(H).max()
    assert np.abs(h1 - proj).max() <= 1e-12 * scale
    if n_orb is None:
        assert np.abs(S.conj().T @ S - np.eye(2 * nb)).max() <= 1e-12
        assert np.abs(np.linalg.eigvalsh(h1) - np.linalg.eigvalsh(H)).max() <= 1e-12 * scale
    # the pin separates the plausible slips
    O = ci_oracle.orbital_overlaps(phi)
    for bad in (O.transpose(0, 3, 2, 1), O.conj(), O.transpose(2, 1, 0, 3)):
        assert np.abs(ci_oracle.one_body(E, bad, p.material["delta_so"]) - proj).max() > 1e-6 * scale


# --------------------------------------------------------------------------
# g-matrices (Sec. III B) and the magnetic two-hole model (Eqs. 16-17)
from oracle import exchange as ex_oracle  # noqa: E402
from oracle import gtensor as gt_oracle  # noqa: E402


def test_g_matrix_free_spin_without_spin_orbit():
    """Delta_so = 0: the 6x6 operator is H0 x 1_spin at B = 0, the lowest
    doublet is phi (real, orbital non-degenerate) times spin, and only the
    spin Zeeman term mu_B B.sigma acts on it (the orbital responses of a
    real state vanish).  In the explicit basis {phi up, phi down} g = 2 I
    exactly; in the eigensolver's basis g^T g = 4 I."""
    p = _box(12, 6, 6, seed=3)
    p.material.update(delta_so=0.0)
    Np = p.n_points
    _, phi = eig.lowest_dense(kp.assemble_h0(p), 1)
    U = np.zeros((6 * Np, 2), dtype=complex)
    U.reshape(Np, 2, 3, 2)[:, 0, :, 0] = phi[:, 0].reshape(Np, 3)
    U.reshape(Np, 2, 3, 2)[:, 1, :, 1] = phi[:, 0].reshape(Np, 3)
    g = gt_oracle.g_matrix(gt_oracle.magnetic_response(p, U))
    assert np.abs(g - 2.0 * np.eye(3)).max() < 1e-9
    _, U2 = gt_oracle.lowest_states(p, 2)
    G, gp = gt_oracle.g_tensor(gt_oracle.g_matrix(gt_oracle.magnetic_response(p, U2)))
    assert np.abs(G - 4.0 * np.eye(3)).max() < 1e-9


@pytest.mark.parametrize("rot", ["identity", "device"])
def test_g_matrix_predicts_the_zeeman_splitting(rot):
    """With spin-orbit coupling and strain, the splitting of the lowest
    Kramers doublet of the full operator H(b n) equals mu_B b |g n| up to
    terms of order b^3 (second-order terms are proportional to the identity
    on a Kramers doublet), for several directions n: an eigenvalue check
    independent of the projection that defines g."""
    p = _box(12, 6, 6, seed=3, rot=rot)
    _, U = gt_oracle.lowest_states(p, 2)
    g = gt_oracle.g_matrix(gt_oracle.magnetic_response(p, U))
    rng = np.random.default_rng(4)
    b = 1e-2
    for n in [np.eye(3)[0], np.eye(3)[2]] + list(rng.standard_normal((2, 3))):
        n = n / np.linalg.norm(n)
        w, _ = eig.lowest_dense(kp.assemble(p.with_(B=b * n)), 2)
        assert abs((w[1] - w[0]) / (kp.MU_B * b) - np.linalg.norm(g @ n)) < 1e-6 * np.abs(g).max()
    # the g-tensor is basis independent: a random U(2) rotation of the doublet
    q, _ = np.linalg.qr(rng.standard_normal((2, 2)) + 1j * rng.standard_normal((2, 2)))
    g2 = gt_oracle.g_matrix(gt_oracle.magnetic_response(p, U @ q))
    assert np.abs(g2.T @ g2 - g.T @ g).max() < 1e-10
    assert abs(np.linalg.det(g2) - np.linalg.det(g)) < 1e-10


@pytest.mark.parametrize("rot", ["identity", "device"])
def test_left_right_g_tensors_mirror_symmetric_double_dot(rot):
    """A double dot symmetric under x -> -x (noise-free double well plus
    x-independent terms that break the y and z mirrors; the {100} and {110}
    mirrors are crystal symmetries) maps the left dot onto the right one.
    B is axial, so G_R = S G_L S with S = diag(1, -1, -1), and the
    off-diagonal G_xy, G_xz flip sign (nonzero here)."""
    p = _box(14, 6, 6, seed=3, strain=False, noise_mev=0.0, rot=rot)
    z, y, x = np.meshgrid(np.arange(p.nz), np.arange(p.ny), np.arange(p.nx), indexing="ij")
    V = p.V + 3e-3 * (y - 2.5) / 6 + 2e-3 * (z - 2.5) / 6 + 1e-3 * (y - 2.5) * (z - 2.5) / 36
    d = gt_oracle.dqd_g_tensors(p.with_(V=V))
    S = np.diag([1.0, -1.0, -1.0])
    GL = d["g_left"].T @ d["g_left"]
    GR = d["g_right"].T @ d["g_right"]
    assert np.abs(GR - S @ GL @ S).max() < 1e-9
    assert np.abs(d["gsym_right"] - S @ d["gsym_left"] @ S).max() < 1e-9
    assert max(abs(GL[0, 1]), abs(GL[0, 2])) > 1e-3
    # the symmetric tensor squares to G and keeps the sign of det g
    assert np.abs(d["gsym_left"] @ d["gsym_left"] - GL).max() < 1e-12
    assert np.sign(np.linalg.det(d["gsym_left"])) == np.sign(np.linalg.det(d["g_left"]))


def test_hb_is_two_spin_zeeman_plus_singlet_tunnelling():
    """Eq. 16 at t = 0: the {S(1,1), T+, T-, T0} block is the two-spin
    Zeeman Hamiltonian b_L.sigma_L + b_R.sigma_R with b_L,R = (bbar +- db)/2
    (spectrum +-|b_L| +- |b_R| for random fields); at zero field the
    singlet block [[U - eps, sqrt2 t], [sqrt2 t, 0]] gives
    ((U - eps) -+ sqrt((U - eps)^2 + 8 t^2)) / 2, and the lower root tends
    to -J = -2 t^2 / (U - eps)."""
    rng = np.random.default_rng(11)
    for _ in range(4):
        bL, bR = rng.standard_normal((2, 3)) * 1e-5
        H = ex_oracle.hamiltonian_b(1e-3, 0.0, bL + bR, bL - bR)
        assert np.abs(H - H.conj().T).max() == 0.0
        a, b = np.linalg.norm(bL), np.linalg.norm(bR)
        assert np.abs(np.linalg.eigvalsh(H[1:, 1:]) - np.sort([a + b, -a - b, a - b, b - a])).max() < 1e-18
        bb = bL + bR
        wt = np.linalg.eigvalsh(ex_oracle.hamiltonian_b(1e-3, 0.0, bb, np.zeros(3))[2:, 2:])
        assert np.abs(wt - np.linalg.norm(bb) * np.array([-1.0, 0.0, 1.0])).max() < 1e-18
    ue, t = 2e-3, 1.13e-5
    w = np.linalg.eigvalsh(ex_oracle.hamiltonian_b(ue, t, np.zeros(3), np.zeros(3)))
    r = np.sqrt(ue * ue + 8 * t * t)
    assert np.abs(w - np.sort([0.0, 0.0, 0.0, (ue - r) / 2, (ue + r) / 2])).max() < 1e-18
    J = 2 * t * t / ue
    assert abs(-(ue - r) / 2 - J) < 1e-3 * J
    assert abs(ex_oracle.u_minus_eps(ex_oracle.tunnel_coupling(np.sqrt(2) * t), J) - ue) < 1e-15


def test_anisotropic_exchange_closed_forms():
    """Isotropic, equal g-tensors, n_so = z: for B along n_so the exchange
    stays isotropic (|J_perp| = J_par = J); for B perpendicular to n_so
    |J_perp| = J cos^2 theta_so and J_par = J cos 2 theta_so; without
    spin-orbit rotation J_perp = J_par = J for any B, and delta E_Z = 0."""
    J, th = 1.0e-6, 0.3
    g = 1.7 * np.eye(3)
    n = np.array([0.0, 0.0, 1.0])
    _, jp, jl, dz = ex_oracle.anisotropic_exchange(J, g, g, th, n, [0.0, 0.0, 0.5])
    assert abs(jp - J) < 1e-15 and abs(jl - J) < 1e-15
    for B in ([0.5, 0.0, 0.0], [0.3, -0.4, 0.0]):
        _, jp, jl, dz = ex_oracle.anisotropic_exchange(J, g, g, th, n, B)
        assert abs(jp - J * np.cos(th) ** 2) < 1e-15 and abs(jl - J * np.cos(2 * th)) < 1e-15
        assert abs(dz - kp.MU_B * 1.7 * 0.5 * np.sin(th)) < 1e-15
    rng = np.random.default_rng(2)
    for B in rng.standard_normal((3, 3)):
        _, jp, jl, dz = ex_oracle.anisotropic_exchange(J, g, g, 0.0, rng.standard_normal(3), B)
        assert abs(jp - J) < 1e-15 and abs(jl - J) < 1e-15 and dz == 0.0


# --------------------------------------------------------------------------
# Anderson mixing of the SP loop (an addition: the paper only iterates to
# convergence)
from oracle import poisson as po_oracle  # noqa: E402


@pytest.mark.parametrize("beta", [1.0, 0.5])
def test_anderson_terminates_on_linear_fixed_point(beta):
    """On a linear map G(V) = A V + c in n dimensions, Anderson mixing with
    unlimited depth is equivalent to GMRES on (I - A) V = c, so it reaches
    the fixed point after at most n + 1 steps in exact arithmetic; linear
    mixing with the same weight is still far from it."""
    rng = np.random.default_rng(3)
    n = 6
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    A = Q @ np.diag(rng.uniform(-0.95, 0.95, n)) @ Q.T
    c = rng.standard_normal(n)
    Vstar = np.linalg.solve(np.eye(n) - A, c)
    acc = po_oracle.Anderson(beta, depth=20)
    V = np.zeros(n)
    lin = np.zeros(n)
    for _ in range(n + 2):
        V = acc.step(V, A @ V + c)
        lin = (1 - beta) * lin + beta * (A @ lin + c)
    assert np.abs(V - Vstar).max() < 1e-9 * np.abs(Vstar).max()
    assert np.abs(lin - Vstar).max() > 1e-3 * np.abs(Vstar).max()


def test_anderson_first_step_is_linear_mixing():
    rng = np.random.default_rng(4)
    V, GV = rng.standard_normal(10), rng.standard_normal(10)
    acc = po_oracle.Anderson(0.3, depth=4)
    assert np.abs(acc.step(V, GV) - (0.7 * V + 0.3 * GV)).max() < 1e-15


# --------------------------------------------------------------------------
# Schroedinger-Poisson loop with relaxed occupations (the reading of the
# paper's "repeated till convergence" at 1.5 K)
def _free_energy(f, e0, K, kT):
    f = np.clip(f, 1e-300, 1 - 1e-16)
    return e0 @ f + 0.5 * f @ K @ f + kT * np.sum(f * np.log(f) + (1 - f) * np.log(1 - f))


def test_relaxed_occupations_without_coupling_are_fermi_dirac():
    rng = np.random.default_rng(21)
    e0 = np.sort(rng.uniform(0.0, 5e-3, 8))
    kT = po_oracle.KB_EV * 4.0
    f, mu, eps = po_oracle.relaxed_occupations(e0, np.zeros((8, 8)), 2.0, kT)
    mu_ref = po_oracle.fermi_level(e0, 2.0, kT)
    assert np.abs(f - po_oracle.occupations(e0, mu_ref, kT)).max() < 1e-12
    assert np.abs(eps - e0).max() == 0.0


@pytest.mark.parametrize("T", [1.5, 20.0])
def test_relaxed_occupations_minimise_the_free_energy(T):
    """The occupations minimise e0.f + f.K.f/2 - T S(f) at fixed hole number
    (K a Coulomb-like positive matrix): every feasible perturbation (sum of
    the changes zero, 0 < f < 1) raises it; and sum f = n_holes."""
    rng = np.random.default_rng(int(T))
    n = 8
    e0 = np.sort(rng.uniform(0.0, 4e-3, n))
    L = rng.standard_normal((n, n))
    K = 2e-3 * (L @ L.T) / n + 3e-3 * np.eye(n)
    kT = po_oracle.KB_EV * T
    f, mu, eps = po_oracle.relaxed_occupations(e0, K, 2.0, kT)
    assert abs(f.sum() - 2.0) < 1e-10
    F0 = _free_energy(f, e0, K, kT)
    for _ in range(200):
        d = rng.standard_normal(n)
        d -= d.mean()
        t = 1e-4 * min(1.0, 0.5 * np.min(np.where(d > 0, (1 - f) / np.abs(d), f / np.abs(d + 1e-300))))
        assert _free_energy(f + t * d, e0, K, kT) >= F0 - 1e-15


def test_relaxed_loop_fixed_point_is_a_plain_fixed_point():
    """Iterated to convergence, the relaxed loop stops at a potential V that
    the plain Schroedinger-Poisson map (Fermi-Dirac occupations of the
    states of H(V), density, Poisson, V_ext + phi) reproduces; the
    Coulomb matrix of the step is symmetric positive semidefinite."""
    p = inputs.small_problem(8, 4, 4, h=0.5, seed=5, strain=False)
    g = np.zeros((p.nz, p.ny, p.nx), dtype=np.uint8)
    g[:, :, 0] = 1
    g[:, :, -1] = 1
    gphi = np.zeros_like(p.V)
    V, E, mu, f, hist = po_oracle.sp_loop_relaxed(p, p.V, g, gphi, 6, 1.0, 1.5, 0.8, 40, anderson_depth=4)
    assert hist[-1] < 1e-11, hist
    q = p.with_(V=V.reshape(p.nz, p.ny, p.nx))
    E2, psi = eig.lowest_dense(kp.assemble(q), 6)
    kT = po_oracle.KB_EV * 1.5
    occ = po_oracle.occupations(E2, po_oracle.fermi_level(E2, 1.0, kT), kT)
    rho = observables.density(psi, occ) / p.h ** 3
    GV = p.V.reshape(-1) + po_oracle.solve(p.nx, p.ny, p.nz, p.h, g, gphi, rho)
    assert np.abs(GV - V).max() < 1e-9
    dens = po_oracle.state_densities(psi)
    Q = np.stack([po_oracle.solve(p.nx, p.ny, p.nz, p.h, g, gphi, dens[j] / p.h ** 3) for j in range(6)])
    K = dens @ Q.T
    assert np.abs(K - K.T).max() < 1e-12 * np.abs(K).max()
    # positive semidefinite (Kramers partners share their density: rank n/2)
    assert np.linalg.eigvalsh(0.5 * (K + K.T)).min() > -1e-12 * np.abs(K).max()


@pytest.mark.parametrize("rot", ["identity", "device"])
def test_g_tensor_of_a_doublet_is_gauge_invariant(rot):
    """A gauge change multiplies H(B) by a unitary phase e^{i chi(B)} with
    chi linear in B, which adds i [dchi/dB, H] to dH/dB; its matrix elements
    between the two states of a degenerate doublet vanish.  So g^T g of the
    lowest doublet is the same in the symmetric and the Landau gauge (to the
    finite-difference terms, ~1e-9 here)."""
    p = _box(12, 6, 6, seed=3, rot=rot)
    Gs = []
    for gauge in (0, 1):
        q = p.with_(gauge=gauge)
        _, U = gt_oracle.lowest_states(q, 2)
        g = gt_oracle.g_matrix(gt_oracle.magnetic_response(q, U))
        Gs.append(g.T @ g)
    assert np.abs(Gs[0] - Gs[1]).max() < 2e-8
    assert np.abs(Gs[0]).max() > 1e-2


def test_tunnel_coupling_reproduces_the_papers_worked_example():
    """Sec. III B quotes t = 1.13e-5 eV from the bonding/anti-bonding
    energies printed with Fig. 3(a) (0.813 and 0.797 meV at zero detuning)
    through t = Delta / sqrt(2) (tests/golden/tunnel_coupling.txt); the
    oracle's t matches to the printed three digits."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "tunnel_coupling.txt")
    vals = {}
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        k, v, _ = line.split()
        vals[k] = float(v)
    delta = abs(vals["E_bonding_eps0"] - vals["E_antibonding_eps0"]) * 1e-3      # eV
    t = ex_oracle.tunnel_coupling(delta)
    assert abs(t - vals["t_printed"]) <= 0.005e-5
    assert f"{t:.2e}" == "1.13e-05"
