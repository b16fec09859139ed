"""CPU-side checks of the C ABI library: it loads, exports every entry point
include/fs.h declares, and validates parameters without touching a GPU."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def fs():
    from paper_2507_14282_gb300 import build
    build.build()
    from paper_2507_14282_gb300 import fs as m
    return m


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "fs.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(fs_[a-z_]+)\s*\(", text)))


def test_library_exports_every_declared_symbol(fs):
    lib = fs.lib()
    names = declared_symbols()
    assert len(names) >= 12
    for n in names:
        assert hasattr(lib, n), n


def test_defaults_and_query(fs):
    p = fs.params_default(1)
    assert p["dim"] == 1 and p["ny"] == 1 and p["r_comp"] == 4.0
    s = fs.query(dim=1, nx=512, ppc=32)
    assert s.device_bytes > 0 and s.device_bytes % s.device_alignment == 0
    assert s.nxn == 513 and s.tiles * s.tile_x == 512
    s2 = fs.query(dim=2, nx=256, ny=64, ppc=16, precision=fs.FS_FP32)
    assert s2.tiles == (256 // s2.tile_x) * (64 // s2.tile_y)
    sp = fs.query(dim=1, nx=64, ppc=8, bc_x=fs.FS_BC_PERIODIC)
    assert sp.nxn == 64


def test_query_scales_with_capacity(fs):
    a = fs.query(dim=1, nx=512, ppc=32, capacity_factor=2.0)
    b = fs.query(dim=1, nx=512, ppc=32, capacity_factor=4.0)
    assert b.device_bytes > a.device_bytes and b.particle_capacity > a.particle_capacity


@pytest.mark.parametrize("bad", [
    dict(dim=3), dict(nx=1), dict(dim=1, ny=4), dict(dt=0.0), dict(dx=-1.0),
    dict(precision=7), dict(ppc=0), dict(n_sub=0), dict(bc_x=5),
    dict(fs_mode_thermal=9), dict(n_floor=0.0), dict(capacity_factor=0.5),
    dict(cr_enable=1, p_iso=1.0, mach_a=10.0), dict(hist_pmin=5.0, hist_pmax=1.0),
    dict(nx=70000), dict(tile_x=3, nx=512),
    dict(push_chunk=700), dict(push_chunk=640), dict(push_ctas_per_sm=-1),
])
def test_query_rejects_bad_parameters(fs, bad):
    kw = dict(dim=1, nx=512, ppc=8)
    kw.update(bad)
    with pytest.raises(fs.FsError) as e:
        fs.query(**kw)
    assert e.value.code == -1


def test_strerror_names(fs):
    assert fs.strerror(0) == "ok"
    assert "capacity" in fs.strerror(-2)
    assert "memory" in fs.strerror(fs.FS_ENOMEM)
    assert fs.strerror(-99) == "unknown status"


def test_oracle_is_not_imported_by_the_package():
    import subprocess
    import sys
    code = ("import sys, paper_2507_14282_gb300; "
            "assert not any(m == 'oracle' or m.startswith('oracle.') for m in sys.modules)")
    subprocess.run([sys.executable, "-c", code], check=True, cwd=ROOT)


def test_window_query_sizes_and_rejections(fs):
    import ctypes as C
    L = fs.lib()

    def q(steps=200, ckpt=20, n=262144, modes=16, **kw):
        kw.setdefault("dim", 1)
        kw.setdefault("ny", 1)
        p = fs.make_params(nx=2048, ppc=128, dt=0.0025, mach_a=20.0, cr_enable=1, **kw)
        b = C.c_size_t()
        rc = L.fs_window_query(C.byref(p), steps, ckpt, n, modes, C.byref(b))
        return rc, b.value

    rc, b32 = q(precision=fs.FS_FP32)
    assert rc == 0 and b32 > 262144 * 16 * 11  # state, ten checkpoints, the tape
    rc, b64 = q(precision=fs.FS_FP64)
    assert rc == 0 and b64 > b32
    assert q(precision=fs.FS_FP32, steps=400)[1] > b32  # more checkpoints
    assert q(dim=2, ny=16)[0] == -1          # 1D only
    assert q(c_light=50.0)[0] == -1          # no relativistic ions
    assert q(bc_x=fs.FS_BC_PERIODIC)[0] == -1
    assert q(steps=0)[0] == -1 and q(ckpt=0)[0] == -1 and q(n=-1)[0] == -1
    # the reverse sweep keeps a tile's RK4 stage inputs in shared memory (at
    # most 227 KB a CTA): FP64 up to 9 substeps, FP32 up to 10
    assert q(precision=fs.FS_FP64, n_sub=9)[0] == 0
    assert q(precision=fs.FS_FP64, n_sub=10)[0] == -1
    assert q(precision=fs.FS_FP32, n_sub=10)[0] == 0
    assert q(precision=fs.FS_FP32, n_sub=11)[0] == -1
    assert q(n_sub=0)[0] == -1


def test_fp64_fma_rate_rejects_bad_arguments(fs):
    # checked before any CUDA call, so this runs without a GPU
    import ctypes as C
    out = C.c_double()
    L = fs.lib()
    assert L.fs_fp64_fma_rate(0, None, C.byref(out)) == -1  # FS_EINVAL
    assert L.fs_fp64_fma_rate((1 << 24) + 1, None, C.byref(out)) == -1  # FS_EINVAL
    assert L.fs_fp64_fma_rate(16, None, None) == -1  # FS_EINVAL


def test_every_entry_point_body_is_guarded():
    # No C++ exception may cross the C ABI: each function fs.h declares is
    # defined with its body inside FS_GUARD_BEGIN ... FS_GUARD_END (fs_strerror
    # only returns string literals)
    csrc = os.path.join(ROOT, "paper_2507_14282_gb300", "csrc")
    text = "".join(open(os.path.join(csrc, f)).read() for f in sorted(os.listdir(csrc))
                   if f.endswith(".cu"))
    for name in declared_symbols():
        if name == "fs_strerror":
            continue
        m = re.search(r"\bint\s+" + name + r"\s*\([^;{]*\)\s*\{", text)
        assert m, f"{name}: definition not found"
        body = text[m.end():m.end() + 400]
        assert body.lstrip().startswith("FS_GUARD_BEGIN"), f"{name} is not guarded"


def test_restore_state_rejects_null_arguments(fs):
    # checked before any CUDA call
    L = fs.lib()
    assert L.fs_restore_state(None, None, 0) == -1


def test_query_accepts_push_launch_shapes(fs):
    # FP32 takes 512- or 576-particle chunks, FP64 512; any CTA cap >= 0
    for prec, chunk in ((fs.FS_FP32, 512), (fs.FS_FP32, 576), (fs.FS_FP64, 512)):
        s = fs.query(dim=2, nx=256, ny=64, ppc=64, precision=prec, push_chunk=chunk,
                     push_ctas_per_sm=2)
        assert s.device_bytes > 0
