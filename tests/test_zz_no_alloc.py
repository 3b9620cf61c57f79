"""The allocation-free residual entry point agrees with hz_residual.

hz_residual_noalloc serves callers that cannot allocate device memory at the
point of the call (memory reserved up front by another allocator, or loops
that forbid allocation calls).  It keeps its scratch in a fixed device array
inside the library.  This test calls it through the C ABI twice in a row and
compares each result with the allocating entry point hz_residual, at the
tolerance the residual parity test uses.  The file is named so that pytest
collects it last.
"""
import ctypes

import numpy as np
import pytest

import hz_inputs as I

pytestmark = pytest.mark.gpu

hz = pytest.importorskip("paper_1510_01831_gb300.hz")


def test_noalloc_residual_matches_hz_residual_twice():
    torch = pytest.importorskip("torch")
    pb = I.smooth_random(60, n_pml=5, L=3, C=2, seed=61, ppw=8, corr_pts=8, n_z=44)
    ctx = hz.Context(pb.m, pb.n_x, pb.n_z, pb.omega, pb.h, pb.n_pml, pb.L, pb.C)
    ctx.hz_factor()
    lib = hz.load()
    rng = np.random.default_rng(62)
    for call in range(2):
        B = 3 + call
        f = I.random_sources(pb.shape_ext, pb.n_pml, B, 63 + call)
        u = (rng.standard_normal(f.shape) + 1j * rng.standard_normal(f.shape)) * 1e-3
        ref = ctx.hz_residual(np.ascontiguousarray(u), f)          # allocating entry point (host arrays)
        u_d = torch.from_numpy(np.ascontiguousarray(u)).cuda()
        f_d = torch.from_numpy(f).cuda()
        res_d = torch.full((B,), -1.0, dtype=torch.float64, device="cuda")
        st = lib.hz_residual_noalloc(ctx._ctx, ctypes.c_void_p(u_d.data_ptr()), ctypes.c_void_p(f_d.data_ptr()), B,
                                     ctypes.c_void_p(res_d.data_ptr()))
        assert st == hz.HZ_OK, lib.hz_last_error(ctx._ctx)
        torch.cuda.synchronize()
        got = res_d.cpu().numpy()
        assert np.allclose(got, ref, rtol=1e-10), (call, got, ref)
    # sizes beyond the preallocated scratch are rejected with a message
    big = torch.zeros((257,) + pb.shape_ext, dtype=torch.complex128, device="cuda")
    r = torch.zeros(257, dtype=torch.float64, device="cuda")
    st = lib.hz_residual_noalloc(ctx._ctx, ctypes.c_void_p(big.data_ptr()), ctypes.c_void_p(big.data_ptr()), 257,
                                 ctypes.c_void_p(r.data_ptr()))
    assert st == hz.HZ_EINVAL
    assert b"256" in lib.hz_last_error(ctx._ctx)
    # host arrays are rejected before any kernel could dereference them
    uh = np.zeros((2,) + pb.shape_ext, complex)
    rh = np.zeros(2)
    st = lib.hz_residual_noalloc(ctx._ctx, ctypes.c_void_p(uh.ctypes.data), ctypes.c_void_p(uh.ctypes.data), 2,
                                 ctypes.c_void_p(rh.ctypes.data))
    assert st == hz.HZ_EINVAL
    assert b"device memory" in lib.hz_last_error(ctx._ctx)
    ctx.close()
