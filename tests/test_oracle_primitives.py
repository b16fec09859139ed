"""Pins of the oracle's building blocks against facts fixed outside the oracle.

Random numbers: Philox4x32-10 (Salmon et al., SC'11) known-answer value and
avalanche/uniformity; the project's own log and sincos against mpmath;
Box-Muller normals against the normal law. Boris rotation against its closed
form; CIC gather against exact bilinear interpolation.
"""
import math

import numpy as np
import pytest
from scipy import stats

from oracle import oracle as O


# ----------------------------------------------------------------- Philox
def test_philox_known_answer_zero_counter():
    # Published known-answer value of Philox4x32-10 for counter 0, key 0.
    out = O.philox([0, 0, 0, 0], [0, 0])
    assert [int(x) for x in out] == [0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8]


def test_philox_avalanche():
    # Ten rounds mix fully: flipping one input bit flips ~half of 128 outputs.
    rng = np.random.default_rng(7)
    flips = []
    for _ in range(64):
        ctr = rng.integers(0, 2**32, 4, dtype=np.uint64).astype(np.uint32)
        key = rng.integers(0, 2**32, 2, dtype=np.uint64).astype(np.uint32)
        base = O.philox(ctr, key)
        for bit in range(0, 128, 7):
            c2 = ctr.copy()
            c2[bit // 32] ^= np.uint32(1 << (bit % 32))
            o2 = O.philox(c2, key)
            flips.append(sum(bin(int(a) ^ int(b)).count("1") for a, b in zip(base, o2)))
    m = np.mean(flips)
    assert abs(m - 64.0) < 1.0, m


def test_philox_uniform_chi2():
    counts = np.zeros(256)
    for pid in range(4096):
        r = O.philox([pid, 3, 1, 0], [12345, 0])
        for w in r:
            counts[int(w) >> 24] += 1
    chi2 = ((counts - counts.mean()) ** 2 / counts.mean()).sum()
    p = stats.chi2.sf(chi2, 255)
    assert p > 1e-3, p


def test_u01_endpoints_exact():
    assert O.u01(0) == 2.0 ** -33
    assert O.u01(2**32 - 1) == 1.0 - 2.0 ** -33
    assert O.u01(2**31) == 0.5 + 2.0 ** -33


# ----------------------------------------------------------------- log, sincos
def _ulp(x):
    return math.ulp(x)


def test_log_accuracy_against_mpmath():
    mp = pytest.importorskip("mpmath")
    mp.mp.prec = 120
    rng = np.random.default_rng(1)
    xs = list(rng.uniform(0, 1, 3000)) + [O.u01(int(k)) for k in
                                          rng.integers(0, 2**32, 3000, dtype=np.uint64)]
    xs += [2.0 ** -33, 0.5, 0.7071067811865476, 0.7071067811865475, 1.4142135623730951,
           1.9999999999, 3.0, 1e3, 1.0 - 2**-53]
    worst = 0.0
    for x in xs:
        exact = float(mp.log(mp.mpf(x)))
        got = O.log(x)
        if exact == 0.0:
            assert got == 0.0
            continue
        worst = max(worst, abs(got - exact) / _ulp(exact))
    assert worst <= 2.0, worst
    assert O.log(1.0) == 0.0
    for k in range(-40, 40):
        assert abs(O.log(2.0 ** k) - k * math.log(2.0)) <= 2 * _ulp(k * math.log(2.0) or 1.0)


def test_sincos2pi_accuracy_against_mpmath():
    mp = pytest.importorskip("mpmath")
    mp.mp.prec = 120
    rng = np.random.default_rng(2)
    us = list(rng.uniform(0, 1, 4000)) + [0.0, 0.125, 0.25, 0.375, 0.5, 0.625, 0.75,
                                           0.875, O.u01(0), O.u01(2**32 - 1)]
    worst = 0.0
    for u in us:
        c, s = O.sincos2pi(u)
        ang = 2 * mp.pi * mp.mpf(u)
        ec, es = float(mp.cos(ang)), float(mp.sin(ang))
        worst = max(worst, abs(c - ec), abs(s - es))
    # absolute error within a few units of 2^-53 on [-1, 1]
    assert worst <= 4 * 2.0 ** -53, worst
    assert O.sincos2pi(0.0) == (1.0, 0.0)


def test_box_muller_normals_from_initial_plasma():
    # Cold-drift-free thermal load: every velocity component is N(0, beta_i/2).
    beta = 2.0
    sim = O.Oracle(dim=1, nx=256, ppc=64, mach_a=0.0, beta_i=beta, bc_x=O.BC_PERIODIC)
    p = sim.particles()
    vth = math.sqrt(beta / 2)
    for comp in ("vx", "vy", "vz"):
        z = p[comp] / vth
        assert abs(z.mean()) < 4 / math.sqrt(z.size)
        assert abs(z.var() - 1.0) < 5 * math.sqrt(2.0 / z.size)
        assert stats.kstest(z, "norm").pvalue > 1e-3
    # positions uniform in the cell
    assert stats.kstest(p["fx"], "uniform").pvalue > 1e-3
    # no correlation between the components
    assert abs(np.corrcoef(p["vx"], p["vy"])[0, 1]) < 4 / math.sqrt(p["vx"].size)


# ----------------------------------------------------------------- Boris
@pytest.mark.parametrize("bmag,dt", [(1.0, 0.005), (3.7, 0.05), (0.2, 0.5)])
def test_boris_rotation_angle_closed_form(bmag, dt):
    # Pure B: Boris rotates v_perp by exactly 2 atan(|B| dt / 2) per step and
    # leaves v_par and |v| unchanged.
    bhat = np.array([0.3, -0.5, 0.8]); bhat /= np.linalg.norm(bhat)
    B = bmag * bhat
    v = np.array([1.0, 2.0, -0.5])
    vpar = v @ bhat
    v1 = O.boris(v, [0, 0, 0], B, dt)
    p0 = v - vpar * bhat; p1 = v1 - (v1 @ bhat) * bhat
    ang = math.atan2(np.linalg.norm(np.cross(p0, p1)), p0 @ p1)
    assert abs(ang - 2 * math.atan(bmag * dt / 2)) < 1e-14
    # gyration sense of a positive charge: rotation about -B
    assert np.cross(p0, p1) @ bhat < 0
    assert abs(v1 @ bhat - vpar) < 1e-14
    assert abs(np.linalg.norm(v1) - np.linalg.norm(v)) < 1e-14


def test_boris_energy_conserved_long_run():
    v = np.array([0.7, -1.1, 0.4]); B = np.array([0.1, 0.9, -0.3])
    e0 = v @ v
    for _ in range(20000):
        v = O.boris(v, [0, 0, 0], B, 0.01)
    assert abs(v @ v - e0) / e0 < 1e-12


def test_boris_exb_drift_fixed_point_and_average():
    # E perpendicular to B: v_d = E x B / B^2 is an exact fixed point of Boris,
    # and a gyrating particle's orbit average is v_d.
    E = np.array([0.0, 0.3, 0.0]); B = np.array([0.0, 0.0, 2.0])
    vd = np.cross(E, B) / (B @ B)
    v = vd.copy()
    for _ in range(1000):
        v = O.boris(v, E, B, 0.01)
    assert np.abs(v - vd).max() < 1e-13
    # gyrating orbit: average over an integer number of discrete periods
    dt = 0.01
    theta = 2 * math.atan(2.0 * dt / 2)
    nper = 2 * math.pi / theta
    nsteps = int(round(20 * nper))
    v = vd + np.array([0.0, 1.0, 0.0])
    acc = np.zeros(3)
    for _ in range(nsteps):
        v = O.boris(v, E, B, dt)
        acc += v
    avg = acc / nsteps
    assert np.abs(avg - vd).max() < 2.0 / nsteps * 5


def test_boris_parallel_electric_kick():
    E = np.array([0.0, 0.0, 0.25]); B = np.array([0.0, 0.0, 1.5])
    v = O.boris([0.0, 0.0, 1.0], E, B, 0.2)
    assert v[2] == pytest.approx(1.0 + 0.25 * 0.2, abs=1e-15)


# ----------------------------------------------------------------- gather
@pytest.mark.parametrize("dim", [1, 2])
def test_cic_gather_reproduces_bilinear_fields(dim):
    nx, ny = 16, (8 if dim == 2 else 1)
    sim = O.Oracle(dim=dim, nx=nx, ny=ny, ppc=1, init_plasma=0, bc_x=O.BC_FAUXSHOCK)
    nxn = sim.nxn
    X, Y = np.meshgrid(np.arange(nxn, dtype=float), np.arange(ny, dtype=float))
    # bilinear in the node coordinates (exact for CIC); y wraps, so test rows
    # j < ny - 1 against the plane and the last row against the wrap
    E = np.stack([0.5 + 0.25 * X - 0.125 * Y + 0.0625 * X * Y,
                  -1.0 + 0.5 * X, 2.0 - 0.75 * Y], axis=-1)
    Bb = np.stack([1.0 + 0 * X, 0.125 * X * Y, -0.25 * X + Y], axis=-1)
    sim.set_node_fields(E, Bb)
    rng = np.random.default_rng(3)
    for _ in range(200):
        i = int(rng.integers(0, nx)); j = int(rng.integers(0, max(ny - 1, 1)))
        fx, fy = rng.uniform(0, 1, 2)
        if dim == 1:
            fy = 0.0
        out = sim.gather(i, j, fx, fy)
        x, y = i + fx, j + fy
        want = np.array([0.5 + 0.25 * x - 0.125 * y + 0.0625 * x * y, -1.0 + 0.5 * x,
                         2.0 - 0.75 * y, 1.0, 0.125 * x * y, -0.25 * x + y])
        if dim == 1:
            want = np.array([0.5 + 0.25 * x, -1.0 + 0.5 * x, 2.0, 1.0, 0.0, -0.25 * x])
        assert np.allclose(out, want, rtol=0, atol=1e-13)
    if dim == 2:
        # top row wraps to row 0
        out = sim.gather(3, ny - 1, 0.0, 1.0 - 2**-53)
        assert np.allclose(out[:3], E[0, 3], atol=1e-12)
