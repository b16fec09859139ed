"""Long-run statistics of the FP32 GPU path against an 8-seed oracle ensemble
(the P12 pin, GPU side).

A FP32 run diverges from any FP64 trajectory within a few hundred steps
(particles that sit within an FP32 ulp of a cell edge move differently), so
after 1000 steps it is one more sample of the same statistics. Its precursor
profiles n(x) and |dB|^2/B0^2(x) and its x-p_x histogram are compared bin by
bin with the ensemble of oracle runs of the same box (1D, 512 cells, 32 ppc,
M_A = 10, seeds 101..108); the run itself uses seed 109.
"""
import numpy as np
import pytest

from tests import ensemble as ens
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


def test_fp32_precursor_profiles_and_phase_space_within_the_oracle_ensemble(fs):
    members = ens.ensemble()
    sim = fs.FauxShock(precision=fs.FS_FP32, **W.scaled(W.CONFIG_1D, seed=109))
    sim.step(ens.STEPS)
    x = ens.observables(sim.grid(fs.FS_PROFILE_N), sim.grid(fs.FS_PROFILE_DB2),
                        sim.histogram())
    d = sim.diag()
    sim.close()
    assert d["status"] == 0
    assert d["incident"] == d["transmitted"] + d["reflected"]
    for k in ("n", "db2", "hist"):
        m = np.array([e[0][k] for e in members])
        frac, zmax = ens.compare(x[k], m, ens.FLOORS[k])
        assert frac >= 0.95 and zmax <= 8.0, (k, frac, zmax)
    # returned fraction of the incident flux: same Eq. 1 statistics
    f_gpu = d["reflected"] / d["incident"]
    f_ens = np.array([e[2]["reflected"] / e[2]["incident"] for e in members])
    assert abs(f_gpu - f_ens.mean()) <= 4.0 * f_ens.std(ddof=1) + 0.01
