"""Host-side checks of the C-ABI library (no GPU needed): it builds for
sm_103a, loads, and exports every function include/khp.h declares; host-side
argument validation answers with the documented status codes."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "khp.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(khp_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2607_08447_b300 import build, _lib
    build.build()
    return _lib.load()


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("khp_create_grid", "khp_set_potential_strain_field", "khp_eigensolve",
                     "khp_density", "khp_eigs_backward", "khp_destroy", "khp_apply",
                     "khp_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name
    assert lib.khp_version() >= 100


def test_binding_covers_every_declared_symbol():
    from paper_2607_08447_b300 import _lib
    assert sorted(_lib.EXPORTED) == _declared()


def test_host_side_validation_without_device(lib):
    from paper_2607_08447_b300 import _lib
    h = ctypes.c_void_p()
    mat = _lib.Material(4.285, 0.339, 1.446, 0.044, -0.42, 2.38, -2.1, -4.85)
    # invalid sizes and spacing are rejected before any CUDA call
    assert lib.khp_create_grid(ctypes.byref(h), 0, 4, 4, 1.0, ctypes.byref(mat), None, None, None) == 1
    assert b"grid sizes" in lib.khp_last_error()
    assert lib.khp_create_grid(ctypes.byref(h), 4, 4, 4, -1.0, ctypes.byref(mat), None, None, None) == 1
    bad_rot = (ctypes.c_double * 9)(1, 0, 0, 0, 2, 0, 0, 0, 1)
    assert lib.khp_create_grid(ctypes.byref(h), 4, 4, 4, 1.0, ctypes.byref(mat), bad_rot, None, None) == 1
    assert b"orthonormal" in lib.khp_last_error()
    # NULL handles
    assert lib.khp_apply(None, None, None, 4, 0) == 1
    assert lib.khp_eigensolve(None, None, None, None, None, None) == 1
    assert lib.khp_destroy(None) == 0


def test_host_side_validation_of_the_next_rows(lib):
    """The entry points of the H0, Poisson/SP, CI and g-tensor rows reject
    NULL handles and out-of-range sizes with INVALID_ARG before any CUDA
    call."""
    from paper_2607_08447_b300 import _lib
    h = ctypes.c_void_p()
    mat = _lib.Material(4.285, 0.339, 1.446, 0.044, -0.42, 2.38, -2.1, -4.85)
    assert lib.khp_create_grid_h0(ctypes.byref(h), 4, 0, 4, 1.0, ctypes.byref(mat), None, None, None) == 1
    buf = (ctypes.c_double * 64)()
    assert lib.khp_position_moments(None, buf, 4, buf) == 1
    assert lib.khp_pair_densities(None, buf, 2, buf) == 1
    assert lib.khp_project_rows(None, buf, None, 8, 2, 0, buf, None) == 1
    P = ctypes.c_void_p()
    assert lib.khp_poisson_create(ctypes.byref(P), 0, 4, 4, 0.5, 11.7, None, None, None) == 1
    assert lib.khp_poisson_create(ctypes.byref(P), 4, 4, 4, 0.5, -1.0, buf, buf, None) == 1
    ch = ctypes.c_double()
    assert lib.khp_sp_update(None, None, buf, 0.5, buf, ctypes.byref(ch)) == 1
    assert lib.khp_sp_anderson(None, None, buf, 0.5, 4, buf, ctypes.byref(ch)) == 1
    assert b"NULL" in lib.khp_last_error()
    assert lib.khp_sp_anderson_reset(None) == 1
    assert lib.khp_poisson_set_preconditioner(None, 1, None) == 1
    assert lib.khp_poisson_solve_many(None, buf, buf, 2, 1, 1e-10, 100, None, None) == 1
    assert lib.khp_poisson_destroy(None) == 0


def test_host_side_validation_of_the_added_calls(lib):
    """khp_filter_step, khp_state_densities, khp_sp_relax_occupations and
    khp_fermi_level reject NULL handles, bad sizes and bad physics
    parameters before any CUDA call."""
    buf = (ctypes.c_double * 64)()
    assert lib.khp_filter_step(None, buf, None, None, None, buf, 8, 0, 8, 1.0, 0.0, 0.0, 1) == 1
    assert lib.khp_state_densities(None, buf, 4, buf) == 1
    mu = ctypes.c_double()
    assert lib.khp_sp_relax_occupations(None, buf, buf, 4, 1.0, 1e-4, buf, None, buf, 1e-12, None, None) == 1
    E = (ctypes.c_double * 4)(0.0, 1e-3, 2e-3, 3e-3)
    assert lib.khp_fermi_level(E, 4, 0.0, 1e-4, ctypes.byref(mu), None) == 1
    assert lib.khp_fermi_level(E, 4, 1.0, 1e-4, ctypes.byref(mu), None) == 0
    assert E[0] < mu.value < E[1] + 0.5e-3
