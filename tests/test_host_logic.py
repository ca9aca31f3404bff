"""Host-side arithmetic of the package (the steps that run on small
matrices on the host) against the oracle's separately written versions,
on random inputs: the Fermi level of the SP loop (the library's
khp_fermi_level, a Newton iteration, against the oracle's bisection), the
spin-orbit block and the Slater-Condon two-hole matrix of the CI, and the
total-spin operator.
No GPU needed."""
import numpy as np
import pytest

from oracle import ci as ci_or
from oracle import kp
from oracle import poisson as po_or
from paper_2607_08447_b300 import ci as ci_pkg
from paper_2607_08447_b300 import poisson as po_pkg


@pytest.fixture(scope="module")
def lib():
    from paper_2607_08447_b300 import _lib, build
    build.build()
    return _lib.load()


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_fermi_level_matches_oracle(lib, seed):
    """The library's Fermi level (safeguarded Newton, khp_fermi_level)
    against the oracle's bisection, which shares no code with it: random
    levels, well separated levels with kT far below the spacing (flat count
    between levels), an exactly degenerate cluster, fractional fillings."""
    rng = np.random.default_rng(seed)
    cases = [np.sort(rng.uniform(-5e-3, 5e-3, 16)),
             np.array([0.0, 1e-3, 2e-3, 5e-3, 9e-3, 2e-2]) + rng.uniform(-1e-2, 1e-2),
             np.array([1e-3, 1e-3, 1e-3 + 1e-9, 4e-3, 4e-3, 8e-3, 8e-3, 1.2e-2])]
    for E in cases:
        for T, nh in ((1.5, 2.0), (20.0, 3.0), (0.3, 1.0), (4.0, 2.5), (1.5, 0.01)):
            kT = 8.617333262e-5 * T
            mu_p, occ = po_pkg.fermi_level(E, nh, kT)
            mu_o = po_or.fermi_level(E, nh, kT)
            f_o = po_or.occupations(E, mu_o, kT)
            # both sides' occupations hold n_holes; mu agrees to the flatness
            # of the count (dN/dmu) times rounding
            assert abs(np.sum(occ) - nh) <= 1e-12 * len(E), (T, nh)
            assert np.abs(occ - f_o).max() <= 1e-10, (T, nh)
            slope = np.sum(f_o * (1 - f_o)) / kT
            assert abs(mu_p - mu_o) <= 1e-12 + 1e-14 * len(E) / slope, (T, nh, mu_p, mu_o)


def test_fermi_level_rejects_bad_input(lib):
    import ctypes
    from paper_2607_08447_b300 import _lib
    E = np.array([0.0, 1e-3, 2e-3])
    mu = ctypes.c_double()
    assert lib.khp_fermi_level(_lib.dptr(E), 3, 3.0, 1e-4, ctypes.byref(mu), None) == 1
    assert lib.khp_fermi_level(_lib.dptr(E), 3, 1.0, 0.0, ctypes.byref(mu), None) == 1
    E[1] = np.inf
    assert lib.khp_fermi_level(_lib.dptr(E), 3, 1.0, 1e-4, ctypes.byref(mu), None) == 1
    assert b"non-finite" in lib.khp_last_error()


def test_spin_orbit_block_matches_oracle():
    for delta in (0.044, 0.3):
        assert np.abs(ci_pkg.spin_orbit_6x6(delta) - kp.spin_orbit_matrix(delta)).max() <= 1e-15


@pytest.mark.parametrize("n", [2, 3, 4])
def test_two_hole_matrix_matches_oracle(n):
    rng = np.random.default_rng(10 + n)
    A = rng.standard_normal((2 * n, 2 * n)) + 1j * rng.standard_normal((2 * n, 2 * n))
    h1 = A + A.conj().T
    J = rng.standard_normal((n, n, n, n)) + 1j * rng.standard_normal((n, n, n, n))
    # the symmetries of Coulomb integrals: particle swap and Hermiticity
    J = J + J.transpose(1, 0, 3, 2)
    J = J + J.transpose(2, 3, 0, 1).conj()
    H_pkg, dets_pkg = ci_pkg._two_hole_matrix(h1, J, n)
    H_or, dets_or = ci_or.ci_matrix(h1, J, n)
    assert list(dets_pkg) == list(dets_or)
    assert np.abs(H_pkg - H_or).max() <= 1e-12 * np.abs(H_or).max()
    S_pkg = ci_pkg._total_spin_squared(n, dets_pkg)
    S_or = ci_or.spin_squared(n)
    assert np.abs(S_pkg - S_or).max() <= 1e-12
