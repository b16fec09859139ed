"""Seeded inputs of the differentiable window (1D faux-shock box): the
initial drifting-Maxwellian plasma, the seeded transverse-B mode amplitudes
and phases, and the parameter vector theta = (a_1..a_M, u_cr, u2). Random
numbers only; none of the method's arithmetic.

The differentiable-window workload: 2048 cells, 128 ppc (262 144 ions),
M_A = 20, theta_Bn = 0, beta = 1, seed 4, 200 steps checkpointed every 20;
16 modes with a_m uniform in +-0.01 B0 and phases uniform in [0, 2 pi); the
cosmic-ray source on with p_iso = 100 and n_cr/n_g = 0.01, drift u_cr and
faux-shock kick u2 = M_A / r = 5. The oracle copy is 64 cells at 8 ppc.
"""
import numpy as np

WINDOW_FULL = dict(nx=2048, ppc=128, steps=200, ckpt=20)
WINDOW_SMALL = dict(nx=64, ppc=8)
COMMON = dict(dx=0.5, dt=0.0025, mach_a=20.0, theta_bn_deg=0.0, beta_i=1.0, beta_e=1.0,
              seed=4)
N_MODES = 16
U_CR, U2 = 5.0, 5.0


def plasma(nx: int, ppc: int, seed: int = 4, mach_a: float = 20.0, beta_i: float = 1.0):
    """Positions in cells (X = i + f, ppc per cell, uniform in the cell) and
    velocities of a Maxwellian of thermal speed sqrt(beta_i/2) drifting at
    -M_A x."""
    rng = np.random.default_rng(seed)
    X = np.repeat(np.arange(nx), ppc) + rng.uniform(0.0, 1.0, nx * ppc)
    V = rng.normal(0.0, np.sqrt(0.5 * beta_i), (nx * ppc, 3))
    V[:, 0] -= mach_a
    return X, V


def modes(seed: int = 4, m: int = N_MODES):
    rng = np.random.default_rng(seed + 1000)
    return rng.uniform(-0.01, 0.01, m), rng.uniform(0.0, 2.0 * np.pi, m)


def theta(amps, u_cr=U_CR, u2=U2):
    return np.concatenate([np.asarray(amps, np.float64), [u_cr, u2]])
