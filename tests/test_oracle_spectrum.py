"""Pins of the oracle's magnetic diagnostics (Sec. 3.1): the transversely
averaged perpendicular power spectrum of the Fig. 3 caption and the y-averaged
lineouts of Fig. 2(b), checked against closed forms, Parseval's identity and a
brute-force DFT."""
import numpy as np
import pytest

from oracle import oracle as O


def field(ny, nx, by, bz, bx=None):
    B = np.zeros((ny, nx, 3))
    B[:, :, 0] = 1.0 if bx is None else bx
    B[:, :, 1] = by
    B[:, :, 2] = bz
    return B


@pytest.mark.parametrize("nx", [64, 96, 250])
def test_single_mode_power_is_a_squared_over_four(nx):
    x = np.arange(nx)
    a, b, m, mz = 0.3, 0.05, 5, 9
    by = a * np.cos(2 * np.pi * m * x / nx + 0.7)
    bz = b * np.sin(2 * np.pi * mz * x / nx)
    P = O.bperp_spectrum(field(4, nx, by, bz))
    assert P.shape == (nx // 2 + 1,)
    assert P[m] == pytest.approx(a * a / 4, rel=1e-12)
    assert P[mz] == pytest.approx(b * b / 4, rel=1e-12)
    rest = np.delete(P, [m, mz])
    assert np.max(rest) < 1e-28


def test_uniform_field_has_only_the_mean_mode():
    P = O.bperp_spectrum(field(3, 32, 0.4, -0.2))
    assert P[0] == pytest.approx(0.4 ** 2 + 0.2 ** 2, rel=1e-14)
    assert np.max(P[1:]) < 1e-30


@pytest.mark.parametrize("nx", [32, 33])
def test_parseval(nx):
    rng = np.random.default_rng(3)
    B = rng.normal(size=(5, nx, 3))
    P = O.bperp_spectrum(B)
    # one-sided spectrum of real rows: k and nx - k carry equal power
    two_sided = P[0] + 2 * P[1:(nx + 1) // 2].sum() + (P[nx // 2] if nx % 2 == 0 else 0.0)
    direct = np.mean(np.sum(B[:, :, 1] ** 2 + B[:, :, 2] ** 2, axis=1)) / nx
    assert two_sided == pytest.approx(direct, rel=1e-12)


def test_brute_force_dft_and_y_average():
    rng = np.random.default_rng(5)
    ny, nx = 3, 12
    B = rng.normal(size=(ny, nx, 3))
    want = np.zeros(nx // 2 + 1)
    for k in range(nx // 2 + 1):
        for j in range(ny):
            for c in (1, 2):
                re = sum(B[j, x, c] * np.cos(2 * np.pi * k * x / nx) for x in range(nx)) / nx
                im = -sum(B[j, x, c] * np.sin(2 * np.pi * k * x / nx) for x in range(nx)) / nx
                want[k] += (re * re + im * im) / ny
    np.testing.assert_allclose(O.bperp_spectrum(B), want, rtol=1e-12, atol=1e-15)


def test_profile_B_is_the_row_mean():
    rng = np.random.default_rng(9)
    B = rng.normal(size=(4, 10, 3))
    prof = O.profile_B(B)
    assert prof.shape == (10, 3)
    for i in range(10):
        for c in range(3):
            assert prof[i, c] == pytest.approx(sum(B[j, i, c] for j in range(4)) / 4, rel=1e-14)
