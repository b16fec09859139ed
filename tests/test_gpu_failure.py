"""Failure detection on the device, exercised without a GPU fault.

Device conditions are sticky bits in a simulation's status word that the
next synchronising call turns into an FS_E* code. These tests reach each
bit through the device path on purpose, in forms that cannot hang or fault:

- a bounded mbarrier wait that runs out (fs_selftest_wait: a barrier nothing
  arrives on, no copy in flight), after which the context stays usable;
- a non-finite field fed from the host (fs_load_fields), which makes the
  push's motion non-finite: FS_ENAN;
- a particle whose cell lies outside its tile, written into the caller-owned
  device buffer: the push's own range check drops it and reports
  FS_EBADCELL.
"""
import numpy as np
import pytest

from oracle import oracle as O
from tests import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fs():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2507_14282_gb300 import build
    build.build()
    from paper_2507_14282_gb300 import fs as m
    return m


def test_bounded_wait_runs_out_and_reports_timeout(fs):
    assert fs.selftest_wait(4096) == fs.FS_ETIMEOUT
    assert fs.selftest_wait(1) == fs.FS_ETIMEOUT
    # the context is still usable: a short FP64 run equals the oracle
    cfg = W.scaled(W.CONFIG_1D, nx=64, ppc=8)
    gpu = fs.FauxShock(precision=fs.FS_FP64, **cfg)
    ref = O.Oracle(**cfg)
    gpu.step(5)
    ref.step(5)
    assert np.array_equal(gpu.grid(fs.FS_B), ref.grid(O.GRID_B))
    assert gpu.diag()["status"] == 0
    gpu.close()


def test_selftest_rejects_bad_arguments(fs):
    import ctypes as C
    L = fs.lib()
    assert L.fs_selftest_wait(0, C.c_void_p(8), None) == -1
    assert L.fs_selftest_wait((1 << 20) + 1, C.c_void_p(8), None) == -1
    assert L.fs_selftest_wait(16, None, None) == -1


def test_non_finite_field_reports_enan(fs):
    sim = fs.FauxShock(precision=fs.FS_FP64, **W.scaled(W.CONFIG_1D, nx=64, ppc=8))
    B = sim.grid(fs.FS_B)
    B[0, 20, 1] = np.nan
    sim.load_fields(B)  # accepted: nothing has moved yet
    sim.step(1)
    with pytest.raises(fs.FsError) as e:
        sim.diag()
    assert e.value.code == fs.FS_ENAN
    with pytest.raises(fs.FsError):  # sticky
        sim.step(1)
    sim.close()


def test_particle_outside_its_tile_reports_ebadcell(fs):
    import torch
    cfg = W.scaled(W.CONFIG_1D, nx=64, ppc=8, tile_x=8)
    sim = fs.FauxShock(precision=fs.FS_FP64, **cfg)
    assert sim.sizes.tiles == 8
    # the device buffer begins with the cell column of particle buffer 0,
    # which holds the particles after fs_init; particle 0 sits in tile 0
    # (cells 0..7). Cell 8 belongs to tile 1.
    off = sim._base - sim._mem.data_ptr()
    col = sim._mem[off:off + 4].view(torch.int32)
    assert 0 <= int(col.item()) < 8
    col.fill_(8)
    sim.step(1)
    with pytest.raises(fs.FsError) as e:
        sim.diag()
    assert e.value.code == fs.FS_EBADCELL
    sim.close()
