"""Seeded synthetic workloads shared by the oracle tests, the GPU parity tests
and the benchmark. Pure parameter sets and input generators: none of the
method's arithmetic lives here.

The paper's runs (Table 1) are 2D boxes with Delta x of order d_i, Delta t a
few 1e-3 / Omega_ci, M_A 20-100; the configurations below have that shape at
sizes one GB300 holds.
"""
import numpy as np

# 1D faux-shock box, FP64 plain method: 512 cells, dx 0.5, 32 ppc, M_A 10,
# theta 0, beta_i = beta_e = 1, dt 0.005, 1000 steps, seed 1
CONFIG_1D = dict(dim=1, nx=512, ny=1, dx=0.5, dy=0.5, dt=0.005, mach_a=10.0,
                 theta_bn_deg=0.0, beta_i=1.0, beta_e=1.0, ppc=32, seed=1)
CONFIG_1D_STEPS = 1000

# 2D production-shaped box, FP64: 4096 x 256, dx 0.5, 16 ppc, M_A 20, theta 0,
# dt 0.0025, seed 2
CONFIG_2D = dict(dim=2, nx=4096, ny=256, dx=0.5, dy=0.5, dt=0.0025, mach_a=20.0,
                 theta_bn_deg=0.0, beta_i=1.0, beta_e=1.0, ppc=16, seed=2)

# 2D precision form, FP32: 8192 x 512, 64 ppc, M_A 30, theta 30 deg,
# dt 0.002, seed 3 (dx not given: 0.5 like the others)
CONFIG_2D_FP32 = dict(dim=2, nx=8192, ny=512, dx=0.5, dy=0.5, dt=0.002, mach_a=30.0,
                      theta_bn_deg=30.0, beta_i=1.0, beta_e=1.0, ppc=64, seed=3)


def scaled(cfg: dict, **kw) -> dict:
    out = dict(cfg)
    out.update(kw)
    return out


def quiet_load(nx, ny, ppc_x, ppc_y=1, vel=None):
    """Evenly spaced particles, ppc_x * ppc_y per cell (a quiet start)."""
    i, j, a, b = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(ppc_x),
                             np.arange(ppc_y), indexing="ij")
    i = i.transpose(1, 0, 2, 3).ravel().astype(np.int32)
    j = j.transpose(1, 0, 2, 3).ravel().astype(np.int32)
    fx = ((a.transpose(1, 0, 2, 3).ravel() + 0.5) / ppc_x)
    fy = ((b.transpose(1, 0, 2, 3).ravel() + 0.5) / ppc_y)
    v = np.zeros((3, i.size)) if vel is None else vel(i + fx, j + fy)
    return i, j, fx, fy, v[0], v[1], v[2]


def random_particles(rng, n, nx, ny, vscale=1.0, drift=0.0):
    """n particles at uniform random positions with Gaussian velocities."""
    ci = rng.integers(0, nx, n).astype(np.int32)
    cj = rng.integers(0, ny, n).astype(np.int32)
    fx = rng.uniform(0, 1, n)
    fy = rng.uniform(0, 1, n)
    v = rng.normal(0, vscale, (3, n))
    v[0] += drift
    return ci, cj, fx, fy, v[0], v[1], v[2]


# Batched ensemble (config 4): 64 independent 1D FP32 runs; run r draws its
# parameters from Philox(key = 100 + r): N_x log-uniform in 512..8192
# (rounded to a multiple of 32 so that tiles divide the box), ppc from
# {32, 64, 128, 256}, M_A uniform in 5..100, theta_Bn uniform in 0..60 deg,
# beta_i = beta_e from {0.5, 1, 2}; dt = min(0.005, 0.1 dx / M_A).
def config4_runs(n_runs: int = 64, first_seed: int = 100, precision: int = 1):
    runs = []
    for r in range(n_runs):
        g = np.random.Generator(np.random.Philox(key=first_seed + r))
        nx = int(round(float(np.exp(g.uniform(np.log(512.0), np.log(8192.0)))) / 32.0)) * 32
        ppc = int(g.choice([32, 64, 128, 256]))
        mach = float(g.uniform(5.0, 100.0))
        theta = float(g.uniform(0.0, 60.0))
        beta = float(g.choice([0.5, 1.0, 2.0]))
        runs.append(dict(dim=1, nx=nx, ny=1, dx=0.5, dy=0.5, dt=min(0.005, 0.1 * 0.5 / mach),
                         mach_a=mach, theta_bn_deg=theta, beta_i=beta, beta_e=beta, ppc=ppc,
                         seed=first_seed + r, precision=precision))
    return runs
