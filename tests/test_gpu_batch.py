"""Batched ensembles on the GPU: independent runs stepped together through
fs_batch_* (one push launch over every run's CTA group, the rest of each
run's step in parallel graph branches) give each run the results of stepping
it alone -- bit-identical in FP64, within the FP32 tolerance in FP32 -- and,
in FP64, the FP64 CPU oracle's results for the same run bit for bit."""
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


RUNS_1D = [
    dict(dim=1, nx=512, ppc=32, mach_a=10.0, theta_bn_deg=0.0, beta_i=1.0, beta_e=1.0,
         dt=0.005, seed=11),
    dict(dim=1, nx=256, ppc=64, mach_a=30.0, theta_bn_deg=40.0, beta_i=0.5, beta_e=0.5,
         dt=0.0016, seed=12, tile_x=4),
    dict(dim=1, nx=1024, ppc=16, mach_a=60.0, theta_bn_deg=20.0, beta_i=2.0, beta_e=2.0,
         dt=0.0008, seed=13, tile_x=64),
    dict(dim=1, nx=96, ppc=128, mach_a=5.0, theta_bn_deg=55.0, beta_i=1.0, beta_e=1.0,
         dt=0.005, seed=14, tile_x=3),
    dict(dim=1, nx=64, ppc=32, mach_a=8.0, theta_bn_deg=10.0, beta_i=1.0, beta_e=1.0,
         dt=0.004, seed=15, bc_x=1),
]
# every run 1D with x walls: the batch runs the whole step tail (movers,
# injection, moments, field advance, step counter) as one launch per kernel
RUNS_1D_WALLS = [r for r in RUNS_1D if r.get("bc_x", 0) == 0]
RUNS_2D = [
    dict(dim=2, nx=64, ny=16, ppc=8, mach_a=10.0, theta_bn_deg=20.0, dt=0.0025, seed=21),
    dict(dim=2, nx=32, ny=8, ppc=16, mach_a=25.0, theta_bn_deg=0.0, dt=0.002, seed=22,
         tile_x=4, tile_y=2),
    dict(dim=2, nx=48, ny=12, ppc=4, mach_a=5.0, theta_bn_deg=45.0, dt=0.004, seed=23),
]


def state(sim, fs):
    p = sim.particles()
    o = np.argsort(p["id"], kind="stable")
    out = {k: v[o] for k, v in p.items()}
    for what, name in ((fs.FS_B, "B"), (fs.FS_E, "E"), (fs.FS_N, "n"), (fs.FS_J, "J")):
        out[name] = sim.grid(what)
    d = sim.diag()
    for k in ("step", "n_particles", "next_id", "incident", "transmitted", "reflected",
              "escaped", "injected", "status"):
        out["diag_" + k] = d[k]
    out["energy"] = np.array([d["kinetic"], d["magnetic"], d["fs_energy"],
                              d["removed_energy"]])
    return out


def run_batched(fs, runs, prec, steps):
    sims = [fs.FauxShock(precision=prec, **r) for r in runs]
    b = fs.FsBatch(sims)
    b.step(1)            # launched directly
    b.step(steps - 1)    # graph replay (both buffer parities)
    batched = [state(s, fs) for s in sims]
    b.close()
    for s in sims:
        s.close()
    return batched


def run_both(fs, runs, prec, steps):
    alone = []
    for r in runs:
        s = fs.FauxShock(precision=prec, **r)
        s.step(steps)
        alone.append(state(s, fs))
        s.close()
    return alone, run_batched(fs, runs, prec, steps)


@pytest.mark.parametrize("runs", [RUNS_1D, RUNS_1D_WALLS, RUNS_2D],
                         ids=["1d", "1d-walls", "2d"])
def test_fp64_batch_is_bit_identical_to_runs_alone(fs, runs):
    alone, batched = run_both(fs, runs, fs.FS_FP64, 12)
    for r, (a, b) in enumerate(zip(alone, batched)):
        assert a["diag_status"] == 0 and b["diag_status"] == 0
        for k in a:
            if k == "energy":
                np.testing.assert_allclose(b[k], a[k], rtol=1e-12, atol=1e-15,
                                           err_msg=f"run {r} {k}")
            elif isinstance(a[k], np.ndarray):
                assert np.array_equal(a[k], b[k]), f"run {r}: {k} differs"
            else:
                assert a[k] == b[k], f"run {r}: {k} {a[k]} != {b[k]}"


def oracle_state(params, steps):
    ref = O.Oracle(**{k: v for k, v in params.items() if k not in ("tile_x", "tile_y")})
    ref.step(steps)
    p = ref.particles()
    o = np.argsort(p["id"], kind="stable")
    out = {k: v[o] for k, v in p.items()}
    for what, name in ((O.GRID_B, "B"), (O.GRID_E, "E"), (O.GRID_N, "n"), (O.GRID_J, "J")):
        out[name] = ref.grid(what)
    d = ref.diag()
    for k in ("step", "n_particles", "next_id", "incident", "transmitted", "reflected",
              "escaped", "injected"):
        out["diag_" + k] = d[k]
    out["energy"] = np.array([d["kinetic"], d["magnetic"], d["fs_energy"],
                              d["removed_energy"]])
    ref.close()
    return out


@pytest.mark.parametrize("runs", [RUNS_1D, RUNS_1D_WALLS, RUNS_2D],
                         ids=["1d", "1d-walls", "2d"])
def test_fp64_batched_runs_equal_the_oracle(fs, runs):
    # every run of a mixed batch (lengths, ppc, M_A, theta, beta, dt, tile
    # shapes, a periodic box) stepped in the batch -- the first step launched
    # directly, the rest replayed from the captured graphs of both buffer
    # parities -- holds the oracle's state of that run, bit for bit
    steps = 12
    batched = run_batched(fs, runs, fs.FS_FP64, steps)
    for r, (params, b) in enumerate(zip(runs, batched)):
        ref = oracle_state(params, steps)
        assert b["diag_status"] == 0
        for k in ref:
            if k == "energy":
                np.testing.assert_allclose(b[k], ref[k], rtol=1e-12, atol=1e-15,
                                           err_msg=f"run {r} {k}")
            elif isinstance(ref[k], np.ndarray):
                assert b[k].shape == ref[k].shape, f"run {r}: {k} shape"
                assert np.array_equal(b[k], ref[k]), f"run {r}: {k} differs from the oracle"
            else:
                assert b[k] == ref[k], f"run {r}: {k} {b[k]} != oracle {ref[k]}"


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(a), 1e-30))


@pytest.mark.parametrize("runs", [RUNS_1D, RUNS_1D_WALLS], ids=["1d", "1d-walls"])
def test_fp32_batch_matches_runs_alone(fs, runs):
    alone, batched = run_both(fs, runs, fs.FS_FP32, 6)
    for r, (a, b) in enumerate(zip(alone, batched)):
        assert a["diag_status"] == 0 and b["diag_status"] == 0
        for k in ("diag_step", "diag_injected", "diag_next_id"):
            assert a[k] == b[k], f"run {r}: {k}"
        assert abs(a["diag_n_particles"] - b["diag_n_particles"]) <= 2
        for k in ("B", "E", "n", "J"):
            assert rel_l2(a[k], b[k]) <= 1e-5, f"run {r}: {k} rel L2 {rel_l2(a[k], b[k])}"


def test_config4_ensemble_steps_with_autotuned_tiles(fs):
    from paper_2507_14282_gb300 import tune
    runs = W.config4_runs(8)
    tuner = tune.Autotuner(probe_particles=1 << 16, warm=2, steps=3)
    tuned = [tuner.tile(r) for r in runs]
    assert all(t["nx"] % t["tile_x"] == 0 for t in tuned)
    assert len(tuner.cache) == len({r["ppc"] for r in runs})
    sims = [fs.FauxShock(**t) for t in tuned]
    n0 = [s.num_particles() for s in sims]
    b = fs.FsBatch(sims)
    b.step(5)
    for s, n in zip(sims, n0):
        d = s.diag()
        assert d["status"] == 0 and d["step"] == 5
        # inflow adds ppc * M_A * dt / dx per step, the wall removes what reaches it
        assert d["n_particles"] == n + d["injected"] - d["transmitted"] - d["escaped"]
    b.close()


def test_autotuner_2d_class_and_launch_shapes(fs):
    # a 2D class: tile shapes, then launch shapes on the winner; the tuned
    # parameters make a valid run, and a batch of such runs equals the oracle
    from oracle import oracle as O
    from paper_2507_14282_gb300 import tune
    tuner = tune.Autotuner(probe_particles=1 << 18, warm=2, steps=3)
    base = dict(dim=2, nx=128, ny=32, ppc=16, mach_a=10.0, theta_bn_deg=20.0, dt=0.0025,
                seed=31, precision=fs.FS_FP64)
    t = tuner.tile(base)
    assert t["nx"] % t["tile_x"] == 0 and t["ny"] % t["tile_y"] == 0
    assert t["push_chunk"] in (0, 512) and t["push_ctas_per_sm"] in (0, 1)
    assert any("tile" in e for e in tuner.log) and any("push_chunk" in e for e in tuner.log)
    runs = [dict(t, seed=31 + k) for k in range(3)]
    sims = [fs.FauxShock(**r) for r in runs]
    b = fs.FsBatch(sims)
    b.step(6)
    for r, s in zip(runs, sims):
        ref = O.Oracle(**{k: v for k, v in r.items()
                          if k not in ("tile_x", "tile_y", "push_chunk", "push_ctas_per_sm",
                                       "precision")})
        ref.step(6)
        assert np.array_equal(s.grid(fs.FS_B), ref.grid(O.GRID_B))
        assert s.diag()["n_particles"] == ref.diag()["n_particles"]
    b.close()


def test_batch_rejects_mixed_precision(fs):
    a = fs.FauxShock(precision=fs.FS_FP64, **RUNS_1D[0])
    c = fs.FauxShock(precision=fs.FS_FP32, **RUNS_1D[1])
    with pytest.raises(fs.FsError):
        fs.FsBatch([a, c])
    a.close()
    c.close()
