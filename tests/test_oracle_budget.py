"""Energy budget of the oracle (kinetic-energy closure, the P11 pin).

Every change of the ions' kinetic energy has one of four causes: the work of
E in the Boris pushes, thermal or cosmic-ray injection, removal at the open
wall or through the faux shock, and the faux-shock return (Sec. 2, Eq. 1),
which keeps the downstream-frame speed but changes the shock-frame energy.
With the oracle's cumulative counters the budget

    K(t) - K(0) = W_push + E_injected - E_removed + E_fs

closes to round-off. Each term is checked to be present, so a dropped term,
a wrong sign or a miscounted removal fails the closure. The magnetic energy
is reported beside it (the isothermal electron fluid is a heat bath, so the
field energy has no closed budget of its own).
"""
import numpy as np
import pytest

from oracle import oracle as o
from tests import workloads as W


def closure(d0, d1):
    rhs = d1["push_work"] + d1["injected_energy"] - d1["removed_energy"] + d1["fs_energy"]
    rhs -= d0["push_work"] + d0["injected_energy"] - d0["removed_energy"] + d0["fs_energy"]
    lhs = d1["kinetic"] - d0["kinetic"]
    return lhs, rhs


def test_kinetic_budget_closes_over_the_1d_faux_shock_run():
    sim = o.Oracle(**W.CONFIG_1D)
    d0 = sim.diag()
    sim.step(400)
    d1 = sim.diag()
    lhs, rhs = closure(d0, d1)
    scale = d1["kinetic"]
    # every term takes part: pushes, inflow, escapes and returns
    assert d1["reflected"] > 0 and d1["escaped"] + d1["transmitted"] > 0
    for k in ("push_work", "injected_energy", "removed_energy", "fs_energy"):
        assert abs(d1[k]) > 1e-6 * scale, k
    assert abs(lhs - rhs) <= 1e-11 * scale, (lhs, rhs)
    # a dropped term breaks it by far more than round-off
    for k in ("push_work", "injected_energy", "removed_energy", "fs_energy"):
        assert abs(lhs - (rhs - d1[k])) > 1e3 * abs(lhs - rhs), k
    assert d1["magnetic"] > 0.0


def test_kinetic_budget_closes_with_cosmic_rays_and_relativistic_ions():
    p = W.scaled(W.CONFIG_1D, nx=128, ppc=16, cr_enable=1, fs_mode_thermal=o.FS_OPEN,
                 n_cr_ratio=0.01, p_iso=20.0, c_light=200.0, seed=11, theta_bn_deg=70.0)
    sim = o.Oracle(**p)
    d0 = sim.diag()
    sim.step(1000)  # oblique B: the cosmic rays gyrate back to the faux shock
    d1 = sim.diag()
    lhs, rhs = closure(d0, d1)
    assert d1["reflected"] > 0 and d1["injected"] > 0
    assert abs(lhs - rhs) <= 1e-11 * d1["kinetic"], (lhs, rhs)


def test_push_work_is_the_energy_gain_in_a_uniform_field():
    # periodic box, no injection, one particle per cell at rest in a fixed
    # E: each gains w v^2 / 2 = push work exactly (up to round-off)
    p = dict(dim=1, nx=8, ny=1, dx=0.5, dt=0.01, mach_a=0.0, bc_x=o.BC_PERIODIC,
             inject_thermal=0, init_plasma=0, ppc=1, beta_e=0.0, seed=3)
    sim = o.Oracle(**p)
    i, j, fx, fy, vx, vy, vz = W.quiet_load(8, 1, 1)
    sim.inject(i, j, fx, fy, vx, vy, vz)
    nxn = sim.nxn
    E = np.zeros((1, nxn, 3))
    E[..., 0] = 0.3
    E[..., 1] = -0.2
    Bb = np.zeros((1, nxn, 3))
    Bb[..., 0] = 1.0
    sim.set_node_fields(E, Bb)
    d0 = sim.diag()
    sim.step(1)
    d1 = sim.diag()
    assert d1["push_work"] > 0
    assert d1["kinetic"] - d0["kinetic"] == pytest.approx(d1["push_work"], rel=1e-12)
