"""GPU parity of the relativistic ions (finite c / v_A, the relativistic
hybrid code of Sec. 2) and of the momentum spectrum n(p), against the FP64
oracle on the same seeded runs: bit-exact FP64 state, exact spectra."""
import numpy as np
import pytest

from oracle import oracle as O
from tests import workloads as W
from tests.test_gpu_parity import assert_state_equal, rel_l2

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


# the paper's two-species set-up with relativistic ions: thermal plasma open
# at the faux shock, cosmic rays injected at it with momentum p_iso
PAPER_1D = dict(dim=1, nx=128, ppc=16, mach_a=8.0, dt=0.004, c_light=25.0, cr_enable=1,
                p_iso=12.0, n_cr_ratio=0.05, fs_mode_thermal=O.FS_OPEN, spec_np=48,
                spec_pmin=0.5, spec_pmax=60.0, seed=41)
PAPER_2D = dict(dim=2, nx=64, ny=16, ppc=8, mach_a=8.0, theta_bn_deg=25.0, dt=0.004,
                c_light=15.0, cr_enable=1, p_iso=10.0, n_cr_ratio=0.05,
                fs_mode_thermal=O.FS_OPEN, spec_np=32, spec_pmin=0.5, spec_pmax=50.0, seed=42)


@pytest.mark.parametrize("cfg,steps", [(PAPER_1D, 60), (PAPER_2D, 25)], ids=["1d", "2d"])
def test_fp64_relativistic_two_species_bit_exact(fs, cfg, steps):
    gpu = fs.FauxShock(precision=fs.FS_FP64, **cfg)
    ref = O.Oracle(**cfg)
    gpu.step(steps)
    ref.step(steps)
    assert_state_equal(gpu, ref, fs)
    for cr in (True, False):
        got = gpu.spectrum_p(cr_only=cr)
        assert np.array_equal(got, ref.spectrum_p(1 if cr else -1)), cr
    assert gpu.spectrum_p(cr_only=True).sum() > 0
    d = gpu.diag()
    # thermal ions reach the open wall and leave; injected CRs stream away
    assert d["incident"] > 0 and d["incident"] == d["transmitted"] + d["reflected"]


def test_fp64_relativistic_fast_cosmic_rays_far_movers(fs):
    # CRs near c cross several cells per step (the far-mover path)
    cfg = dict(PAPER_1D, nx=64, ppc=8, c_light=40.0, p_iso=400.0, dt=0.02, seed=43,
               spec_pmax=2000.0)
    gpu = fs.FauxShock(precision=fs.FS_FP64, **cfg)
    ref = O.Oracle(**cfg)
    gpu.step(20)
    ref.step(20)
    assert_state_equal(gpu, ref, fs)
    assert np.array_equal(gpu.spectrum_p(True), ref.spectrum_p(1))


def test_fp32_relativistic_within_tolerance(fs):
    gpu = fs.FauxShock(precision=fs.FS_FP32, **PAPER_1D)
    ref = O.Oracle(**PAPER_1D)
    gpu.step(1)
    ref.step(1)
    for gw, ow in ((fs.FS_B, O.GRID_B), (fs.FS_N, O.GRID_N), (fs.FS_J, O.GRID_J)):
        assert rel_l2(gpu.grid(gw), ref.grid(ow)) <= 1e-5, gw
    dg, dr = gpu.diag(), ref.diag()
    assert dg["n_particles"] == dr["n_particles"] and dg["injected"] == dr["injected"]
    # spectra agree but for particles within FP32 rounding of a bin edge
    a, b = gpu.spectrum_p(False), ref.spectrum_p(-1)
    assert np.abs(a - b).sum() <= 4


def test_relativistic_batch_matches_runs_alone(fs):
    runs = [dict(PAPER_1D, seed=51), dict(PAPER_1D, nx=96, c_light=12.0, seed=52, tile_x=4)]
    alone = []
    for r in runs:
        s = fs.FauxShock(precision=fs.FS_FP64, **r)
        s.step(10)
        alone.append((s.grid(fs.FS_B), s.spectrum_p(True), s.diag()["reflected"]))
        s.close()
    sims = [fs.FauxShock(precision=fs.FS_FP64, **r) for r in runs]
    b = fs.FsBatch(sims)
    b.step(10)
    for s, (B, sp, refl) in zip(sims, alone):
        assert np.array_equal(s.grid(fs.FS_B), B)
        assert np.array_equal(s.spectrum_p(True), sp)
        assert s.diag()["reflected"] == refl
    b.close()
