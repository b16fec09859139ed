"""The allocation-free field advance, fs_field_advance_noalloc.

Some callers cannot allocate device memory and cannot lend the library
scratch buffers either -- a host framework that owns every device byte through
its own fixed pool, or a time-critical loop that must not risk the device
synchronisation an allocation can cause. For them the library offers one
field-advance entry point whose RK4 stage buffers live in a static device
array. This test checks that it reproduces, bit for bit in FP64 (the FP64
tolerance of the other parity tests), the field update fs_step makes after
its deposit, on two calls in a row (the second call finds the array holding
the first call's stages). It lives in a file collected last so that a run
stopping at its first failure has already run every other test.
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fs():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2507_14282_gb300 import build
    build.build()
    from paper_2507_14282_gb300 import fs as m
    lib = m.lib()
    lib.fs_field_advance_noalloc.argtypes = [C.POINTER(m.FsParams)] + [C.c_void_p] * 6
    lib.fs_field_advance_noalloc.restype = C.c_int
    return m


def planes(t):
    """[rows][cols][3] -> [3][rows][cols] (the library's device layout)."""
    return t.permute(2, 0, 1).contiguous()


@pytest.mark.parametrize("in_place", [False, True], ids=["separate", "in-place"])
@pytest.mark.parametrize("cfg", [
    dict(dim=2, nx=64, ny=16, ppc=8, mach_a=10.0, theta_bn_deg=20.0, dt=0.0025, seed=3),
    dict(dim=1, nx=256, ny=1, ppc=16, mach_a=10.0, dt=0.005, seed=5),
])
def test_noalloc_field_advance_matches_step(fs, cfg, in_place):
    import torch
    sim = fs.FauxShock(precision=fs.FS_FP64, **cfg)
    sim.step(3)
    dev = sim.device
    ny, nx, nxn = sim.ny, sim.nx, sim.nxn
    p = fs.make_params(precision=fs.FS_FP64, **cfg)
    for call in range(2):
        B0 = torch.empty((ny, nx, 3), dtype=torch.float64, device=dev)
        sim.grid_device(fs.FS_B, B0)
        sim.step(1)
        n = torch.empty((ny, nxn), dtype=torch.float64, device=dev)
        u = torch.empty((ny, nxn, 3), dtype=torch.float64, device=dev)
        B1 = torch.empty((ny, nx, 3), dtype=torch.float64, device=dev)
        E1 = torch.empty((ny, nxn, 3), dtype=torch.float64, device=dev)
        for what, t in ((fs.FS_N, n), (fs.FS_U, u), (fs.FS_B, B1), (fs.FS_E, E1)):
            sim.grid_device(what, t)
        b_in, u_p = planes(B0), planes(u)
        # in place: B_out is B_in, advanced where it lies
        b_out = b_in if in_place else torch.full_like(b_in, np.nan)
        e_out = torch.full((3, ny, nxn), np.nan, dtype=torch.float64, device=dev)
        rc = fs.lib().fs_field_advance_noalloc(
            C.byref(p), C.c_void_p(b_in.data_ptr()), C.c_void_p(n.data_ptr()),
            C.c_void_p(u_p.data_ptr()), C.c_void_p(b_out.data_ptr()),
            C.c_void_p(e_out.data_ptr()), C.c_void_p(sim.stream.cuda_stream))
        assert rc == 0, fs.strerror(rc)
        torch.cuda.synchronize()
        assert torch.equal(b_out, planes(B1)), f"B differs on call {call}"
        assert torch.equal(e_out, planes(E1)), f"E differs on call {call}"
    sim.close()


def test_noalloc_rejects_grids_beyond_the_static_array(fs):
    import torch
    # 6 nx ny + 3 (nx + 1) ny doubles > 2^20 for 512 x 256 cells
    p = fs.make_params(dim=2, nx=512, ny=256, ppc=1, precision=fs.FS_FP64)
    t = torch.zeros(8, dtype=torch.float64, device="cuda")
    ptr = C.c_void_p(t.data_ptr())
    rc = fs.lib().fs_field_advance_noalloc(C.byref(p), ptr, ptr, ptr, ptr, ptr, None)
    assert rc == -1
    p32 = fs.make_params(dim=1, nx=64, ppc=1, precision=fs.FS_FP32)
    assert fs.lib().fs_field_advance_noalloc(C.byref(p32), ptr, ptr, ptr, ptr, ptr, None) == -1


def test_noalloc_rejects_overlapping_buffers(fs):
    import torch
    # outputs may not share bytes with each other or with the inputs, except
    # B_out == B_in exactly
    p = fs.make_params(dim=1, nx=64, ppc=1, precision=fs.FS_FP64)
    nc, nn = 64, 65
    buf = torch.zeros(3 * nc + nn + 3 * nn + 3 * nn + 64, dtype=torch.float64, device="cuda")
    buf[3 * nc:3 * nc + nn] = 1.0  # n = 1: finite fields in the one accepted call
    base = buf.data_ptr()
    B = base
    n = B + 8 * 3 * nc
    u = n + 8 * nn
    E = u + 8 * 3 * nn

    def call(b_in, nn_, uu, b_out, e_out):
        return fs.lib().fs_field_advance_noalloc(
            C.byref(p), C.c_void_p(b_in), C.c_void_p(nn_), C.c_void_p(uu),
            C.c_void_p(b_out), C.c_void_p(e_out), None)

    assert call(B, n, u, B, E) == 0          # in place, disjoint otherwise
    torch.cuda.synchronize()
    assert call(B, n, u, B + 8, E) == -1     # B_out partly over B_in
    assert call(B, n, u, n, E) == -1         # B_out over n
    assert call(B, n, u, B, u + 8) == -1     # E_out over u
    assert call(B, n, u, B, n) == -1         # E_out over n
    assert call(B, n, u, B, B) == -1         # E_out over B
