"""Pins of the oracle's relativistic ions (the relativistic hybrid code of
Sec. 2, finite c / v_A) and of the momentum spectrum n(p): Boris rotation
angle and |u| invariance, the non-relativistic limit, free acceleration,
E x B drift, relativistic energies and the spectrum's brute-force binning."""
import numpy as np
import pytest

from oracle import oracle as O


def test_pure_B_rotation_keeps_u_and_turns_by_the_relativistic_angle():
    c = 10.0
    u = np.array([7.0, 0.0, 2.0])  # gamma = sqrt(1 + 53/100)
    B = np.array([0.0, 0.0, 1.3])
    dt = 0.01
    gamma = np.sqrt(1 + u @ u / c ** 2)
    step_angle = 2 * np.arctan(np.linalg.norm(B) * dt / (2 * gamma))
    w = u.copy()
    for _ in range(500):
        w = O.boris_rel(w, [0, 0, 0], B, dt, c)
    assert np.linalg.norm(w) == pytest.approx(np.linalg.norm(u), rel=1e-13)
    assert w[2] == pytest.approx(u[2], abs=1e-13)  # parallel momentum untouched
    ang = np.arctan2(-w[1], w[0])  # rotation sense of q = +1 about +z
    want = (500 * step_angle + np.pi) % (2 * np.pi) - np.pi
    assert ang == pytest.approx(want, abs=1e-10)


def test_large_c_is_the_non_relativistic_push_bit_for_bit():
    rng = np.random.default_rng(1)
    for _ in range(50):
        v, E, B = rng.normal(size=3) * 5, rng.normal(size=3), rng.normal(size=3)
        a = O.boris_rel(v, E, B, 0.01, 1.0e9)  # gamma rounds to 1
        b = O.boris(v, E, B, 0.01)
        assert np.array_equal(a, b)


def test_free_acceleration_is_linear_in_u_and_v_stays_below_c():
    c = 5.0
    u = np.zeros(3)
    E = np.array([2.0, 0.0, 0.0])
    for n in range(1, 2001):
        u = O.boris_rel(u, E, [0, 0, 0], 0.01, c)
    assert u[0] == pytest.approx(2.0 * 0.01 * 2000, rel=1e-12)
    v = u[0] / np.sqrt(1 + u[0] ** 2 / c ** 2)
    assert v < c and v == pytest.approx(c * 40 / np.sqrt(c * c + 1600), rel=1e-12)


def test_relativistic_ExB_drift():
    c = 10.0
    E = np.array([0.0, 3.0, 0.0])
    B = np.array([0.0, 0.0, 1.0])  # E x B / B^2 = (3, 0, 0): 0.3 c
    u = np.zeros(3)
    dt = 0.002
    xs = []
    for _ in range(200000):
        u = O.boris_rel(u, E, B, dt, c)
        g = np.sqrt(1 + u @ u / c ** 2)
        xs.append(u[0] / g)
    # orbit-averaged drift over ~45 gyrations (gyration speed 0.3 c about the
    # drift: the window's partial period bounds the error at about 1%)
    assert np.mean(xs[50000:]) == pytest.approx(3.0, rel=2e-2)


def run(**kw):
    base = dict(dim=1, nx=64, ppc=16, mach_a=5.0, dt=0.005, c_light=20.0, cr_enable=1,
                p_iso=8.0, fs_mode_thermal=O.FS_OPEN, spec_np=40, spec_pmin=0.5,
                spec_pmax=50.0, seed=9)
    base.update(kw)
    return O.Oracle(**base)


def test_relativistic_energy_and_momenta_in_diagnostics():
    sim = run()
    sim.step(20)
    p = sim.particles()
    d = sim.diag()
    c = 20.0
    u2 = p["vx"] ** 2 + p["vy"] ** 2 + p["vz"] ** 2
    g = np.sqrt(1 + u2 / c ** 2)
    w = np.where(p["id"] & O.ID_CR, 0.01 / 16, 1 / 16)
    ke = np.sum(w * (u2 / (g + 1))) * 0.5
    assert d["kinetic"] == pytest.approx(ke, rel=1e-12)
    assert d["incident"] == d["transmitted"] + d["reflected"]
    sim.close()


def test_momentum_spectrum_matches_brute_force_binning():
    sim = run()
    sim.step(30)
    p = sim.particles()
    pm = np.sqrt(p["vx"] ** 2 + p["vy"] ** 2 + p["vz"] ** 2)
    edges = 0.5 * np.exp((np.arange(41) / 40.0) * np.log(50.0 / 0.5))
    cr = (p["id"] & O.ID_CR) != 0
    want_cr = np.histogram(pm[cr], bins=edges)[0]
    want_all = np.histogram(pm, bins=edges)[0]
    got_cr, got_all = sim.spectrum_p(1), sim.spectrum_p(-1)
    assert np.sum(got_cr) > 0
    assert np.array_equal(got_cr, want_cr)
    assert np.array_equal(got_all, want_all)
    # injected CRs carry |u'| = p_iso in the downstream frame: the CR spectrum
    # peaks within a bin or two of p_iso
    k_iso = int(np.searchsorted(edges, 8.0) - 1)
    assert abs(int(np.argmax(got_cr)) - k_iso) <= 2
    sim.close()


def test_non_relativistic_limit_of_a_run():
    a = run(c_light=1.0e7)
    b = run(c_light=0.0)
    a.step(10)
    b.step(10)
    pa, pb = a.particles(), b.particles()
    oa, ob = np.argsort(pa["id"]), np.argsort(pb["id"])
    assert np.array_equal(pa["id"][oa], pb["id"][ob])
    np.testing.assert_allclose(pa["vx"][oa], pb["vx"][ob], rtol=1e-9, atol=1e-9)
    np.testing.assert_allclose(a.grid(O.GRID_B), b.grid(O.GRID_B), rtol=1e-9, atol=1e-11)
    a.close()
    b.close()
