"""GPU parity of the magnetic diagnostics (Sec. 3.1): the transversely
averaged perpendicular power spectrum (shared-memory FFT for power-of-two
rows up to 8192 cells, direct DFT otherwise) and the y-averaged B lineouts,
against the oracle's numpy formulation on the same seeded field."""
import numpy as np
import pytest

from oracle import oracle as O

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


def seeded_field(ny, nx, seed):
    """B0 plus random noise plus a few transverse modes (the shape of a
    Bell-unstable precursor)."""
    rng = np.random.default_rng(seed)
    x = np.arange(nx)
    B = np.zeros((ny, nx, 3))
    B[:, :, 0] = 0.87
    B[:, :, 1] = 0.5 + 0.02 * rng.normal(size=(ny, nx))
    B[:, :, 2] = 0.02 * rng.normal(size=(ny, nx))
    for m, a in ((3, 0.3), (17, 0.1), (nx // 4, 0.05)):
        ph = rng.uniform(0, 2 * np.pi, size=(ny, 1))
        B[:, :, 1] += a * np.cos(2 * np.pi * m * x / nx + ph)
        B[:, :, 2] += a * np.sin(2 * np.pi * m * x / nx + ph)
    return B


CASES = [
    dict(dim=2, nx=256, ny=8, prec=0, why="FFT, FP64"),
    dict(dim=1, nx=96, ny=1, prec=0, why="DFT (not a power of two), FP64"),
    dict(dim=1, nx=8192, ny=1, prec=0, why="largest FFT row, FP64"),
    dict(dim=2, nx=128, ny=4, prec=1, why="FFT, FP32 field"),
    dict(dim=2, nx=8192, ny=4, prec=1, why="largest FFT row, FP32 field"),
    dict(dim=2, nx=12000, ny=2, prec=0, why="DFT longer than the FFT limit"),
]


@pytest.mark.parametrize("case", CASES, ids=[c["why"] for c in CASES])
def test_spectrum_and_lineouts_match_oracle(fs, case):
    nx, ny, dim = case["nx"], case["ny"], case["dim"]
    B = seeded_field(ny, nx, seed=nx + ny)
    if case["prec"] == 1:
        B = B.astype(np.float32).astype(np.float64)  # what an FP32 run holds
    kw = dict(dim=dim, nx=nx, ny=ny, ppc=1, precision=case["prec"])
    if dim == 1:
        kw["theta_bn_deg"] = 30.0
    sim = fs.FauxShock(**kw)
    sim.load_fields(B)
    got = sim.grid(fs.FS_SPECTRUM_BPERP)
    want = O.bperp_spectrum(B)
    assert got.shape == want.shape
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-12 * want.max())
    # the modes put in stand out at their wavenumbers
    for m in (3, 17):
        assert got[m] > 100 * np.median(got)
    prof = sim.grid(fs.FS_PROFILE_B)
    np.testing.assert_allclose(prof, O.profile_B(B), rtol=1e-13, atol=1e-15)
    sim.close()


def test_spectrum_after_steps_matches_oracle_run(fs):
    """After a few steps of a 2D FP64 run, the GPU spectrum and lineouts of
    the run's own field equal the oracle's diagnostics of the oracle's run on
    the same seeded configuration (the FP64 fields themselves are bit-exact)."""
    cfg = dict(dim=2, nx=128, ny=16, ppc=8, mach_a=10.0, theta_bn_deg=20.0, dt=0.0025,
               seed=7)
    sim = fs.FauxShock(precision=0, **cfg)
    sim.step(5)
    ref = O.Oracle(**cfg)
    ref.step(5)
    B = ref.grid(O.GRID_B)
    want = O.bperp_spectrum(B)
    np.testing.assert_allclose(sim.grid(fs.FS_SPECTRUM_BPERP), want, rtol=0,
                               atol=1e-12 * want.max())
    np.testing.assert_allclose(sim.grid(fs.FS_PROFILE_B), O.profile_B(B), rtol=1e-13,
                               atol=1e-15)
    ref.close()
    sim.close()
