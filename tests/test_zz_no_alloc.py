"""The allocation-free backward entry point (khp_eigs_backward_noalloc).

It is for callers that cannot let a library allocate device memory during a
call (all memory owned by a pooling allocator, latency-critical loops where
an allocation could synchronise the device).  Its results must equal those of
khp_eigs_backward on the same inputs, on consecutive calls that reuse its
fixed scratch array.  This file is collected last so that a stop-at-first-
failure run has executed every other test before it.
"""
import ctypes

import numpy as np
import pytest
import torch

import inputs

pytestmark = pytest.mark.gpu


def _call(lib, fn, grid, V, ev, g, levers_t, ng, want_strain=True):
    n = V.shape[1]
    dV = torch.empty(grid.np_, dtype=torch.float64, device="cuda")
    dS = torch.empty(6 * grid.np_, dtype=torch.float64, device="cuda") if want_strain else None
    da = np.zeros(max(ng, 1))
    ev = np.ascontiguousarray(ev, dtype=np.float64)
    g = np.ascontiguousarray(g, dtype=np.float64)
    dp = ctypes.POINTER(ctypes.c_double)
    st = getattr(lib, fn)(grid.handle, ctypes.c_void_p(V.data_ptr()), ev.ctypes.data_as(dp), n,
                          g.ctypes.data_as(dp), ctypes.c_void_p(dV.data_ptr()),
                          None if dS is None else ctypes.c_void_p(dS.data_ptr()),
                          None if levers_t is None else ctypes.c_void_p(levers_t.data_ptr()), ng,
                          da.ctypes.data_as(dp))
    torch.cuda.synchronize()
    return st, dV.cpu().numpy(), (None if dS is None else dS.cpu().numpy()), da[:ng]


def test_noalloc_backward_matches_allocating_entry_point(khp):
    from paper_2607_08447_b300 import _lib
    lib = _lib.load()
    p = inputs.small_problem(11, 9, 7, h=0.5, seed=21, rot="device", strain=True, levers=5)
    grid = khp.KPGrid.from_problem(p)
    levers_t = torch.from_numpy(np.ascontiguousarray(p.levers.reshape(5, -1))).cuda()
    V = torch.from_numpy(inputs.random_block(p.n_unknowns, 6, seed=31)).cuda().contiguous()
    ev = np.array([0.0, 0.1, 0.2, 0.3, 0.4, 0.5])
    for call, g in enumerate(([1.0, -0.5, 2.0, 0.25, 3.0, -1.0], [0.3, 0.3, -4.0, 1.5, 0.0, 2.5])):
        s0, dV0, dS0, da0 = _call(lib, "khp_eigs_backward", grid, V, ev, g, levers_t, 5)
        s1, dV1, dS1, da1 = _call(lib, "khp_eigs_backward_noalloc", grid, V, ev, g, levers_t, 5)
        assert s0 == 0 and s1 == 0, (call, s0, s1)
        assert np.abs(dV1 - dV0).max() <= 1e-12 * np.abs(dV0).max()
        assert np.abs(dS1 - dS0).max() <= 1e-12 * np.abs(dS0).max()
        assert np.abs(da1 - da0).max() <= 1e-12 * np.abs(da0).max()
    # the shared scratch after a larger call: 16 gates, then 3, then none
    # (and no strain output), each against the allocating entry point
    lev16 = torch.from_numpy(inputs.random_block(16, grid.np_, seed=41).real.copy()).cuda().contiguous()
    g = [0.7, -0.2, 1.1, 0.4, -2.0, 0.9]
    for ng, want in ((16, True), (3, True), (0, False)):
        lv = lev16[:ng].contiguous() if ng else None
        s0, dV0, dS0, da0 = _call(lib, "khp_eigs_backward", grid, V, ev, g, lv, ng, want)
        s1, dV1, dS1, da1 = _call(lib, "khp_eigs_backward_noalloc", grid, V, ev, g, lv, ng, want)
        assert s0 == 0 and s1 == 0, (ng, s0, s1)
        assert np.abs(dV1 - dV0).max() <= 1e-12 * np.abs(dV0).max()
        if want:
            assert np.abs(dS1 - dS0).max() <= 1e-12 * np.abs(dS0).max()
        if ng:
            assert np.abs(da1 - da0).max() <= 1e-12 * np.abs(da0).max()
    assert lib.khp_last_error() == b""
    # non-finite dL/dE (Inf as well as NaN) is rejected like the allocating call
    for bad in (np.inf, -np.inf, np.nan):
        gb = [1.0, bad, 0.0, 0.0, 0.0, 0.0]
        st0, *_ = _call(lib, "khp_eigs_backward", grid, V, ev, gb, None, 0, False)
        st1, *_ = _call(lib, "khp_eigs_backward_noalloc", grid, V, ev, gb, None, 0, False)
        assert st0 == 1 and st1 == 1, (bad, st0, st1)
    # gates beyond the fixed scratch are rejected with a clear error
    many = torch.zeros((17, grid.np_), dtype=torch.float64, device="cuda")
    st, *_ = _call(lib, "khp_eigs_backward_noalloc", grid, V, ev, [1.0] * 6, many, 17)
    assert st == 1
    assert b"max 16" in lib.khp_last_error()
    grid.close()
