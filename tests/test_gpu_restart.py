"""Checkpoint / restart: a run saved after N steps and restored into a fresh
handle continues as the straight run of N + M steps does.

Saved: every particle with its id, B at the cell centres, and the run state
(fs_moments(FS_STATE): step counter, next particle number, flux counters,
energy sums, inflow row accumulators). Restored: init_plasma = 0, then
fs_load_fields, fs_inject with the saved ids, fs_restore_state. FP64: every
field, moment, particle and counter bit for bit (the deposit sums are int64
fixed point and do not depend on the particles' order inside a tile; the
random draws are keyed on particle id and step); energy sums to 1e-12 (their
later FP64 atomic additions are order dependent). FP32: within the FP32
field tolerance (its deposit sums are order dependent).
"""
import numpy as np
import pytest

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


def by_id(p):
    o = np.argsort(p["id"], kind="stable")
    return {k: v[o] for k, v in p.items()}


GRID_NAMES = ("B", "E", "BBAR", "N", "J", "U")


def snapshot(sim, fs):
    out = {name: sim.grid(getattr(fs, "FS_" + name)) for name in GRID_NAMES}
    out["particles"] = by_id(sim.particles())
    out["diag"] = sim.diag()
    out["hist"] = sim.histogram()
    return out


CASES = {
    "1d-config": (W.CONFIG_1D, 37, 23),
    "2d-fs-return": (W.scaled(W.CONFIG_2D, nx=64, ny=16, ppc=8, mach_a=10.0,
                              theta_bn_deg=20.0), 11, 9),
    "1d-cosmic-rays": (W.scaled(W.CONFIG_1D, nx=128, fs_mode_thermal=0, cr_enable=1,
                                p_iso=40.0), 60, 40),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_fp64_restart_continues_bit_for_bit(fs, case):
    cfg, n1, n2 = CASES[case]
    straight = fs.FauxShock(precision=fs.FS_FP64, **cfg)
    straight.step(n1 + n2)
    want = snapshot(straight, fs)
    straight.close()

    first = fs.FauxShock(precision=fs.FS_FP64, **cfg)
    first.step(n1)
    ck = first.checkpoint()
    st = fs.FauxShock.run_state_fields(ck["state"])
    assert st["step"] == n1 and st["ny"] == cfg.get("ny", 1)
    first.close()

    again = fs.FauxShock.restart(ck, precision=fs.FS_FP64, **cfg)
    assert again.diag()["step"] == n1
    again.step(1)   # launched directly
    again.step(n2 - 1)  # graph replay
    got = snapshot(again, fs)
    again.close()

    for name in GRID_NAMES:
        assert np.array_equal(got[name], want[name]), name
    assert np.array_equal(got["hist"], want["hist"])
    pg, pw = got["particles"], want["particles"]
    assert pg["id"].size == pw["id"].size
    for k in ("id", "ci", "cj", "fx", "fy", "vx", "vy", "vz"):
        assert np.array_equal(pg[k], pw[k]), k
    dg, dw = got["diag"], want["diag"]
    for k in ("step", "n_particles", "next_id", "incident", "transmitted", "reflected",
              "escaped", "injected", "status"):
        assert dg[k] == dw[k], (k, dg[k], dw[k])
    for k in ("kinetic", "magnetic", "fs_energy", "injected_energy", "removed_energy"):
        assert dg[k] == pytest.approx(dw[k], rel=1e-12, abs=1e-12), k


def test_fp32_restart_within_tolerance(fs):
    cfg = W.scaled(W.CONFIG_2D_FP32, nx=64, ny=16)
    straight = fs.FauxShock(precision=fs.FS_FP32, **cfg)
    straight.step(12)
    first = fs.FauxShock(precision=fs.FS_FP32, **cfg)
    first.step(6)
    again = fs.FauxShock.restart(first.checkpoint(), precision=fs.FS_FP32, **cfg)
    first.close()
    again.step(6)
    for name in GRID_NAMES:
        a = again.grid(getattr(fs, "FS_" + name))
        b = straight.grid(getattr(fs, "FS_" + name))
        assert np.linalg.norm(a - b) <= 1e-5 * np.linalg.norm(b), name
    da, db = again.diag(), straight.diag()
    for k in ("step", "injected", "next_id"):
        assert da[k] == db[k], k
    assert abs(da["n_particles"] - db["n_particles"]) <= 2
    again.close()
    straight.close()


def test_restore_state_rejects_bad_input(fs):
    sim = fs.FauxShock(precision=fs.FS_FP64, **W.scaled(W.CONFIG_1D, nx=64, ppc=8))
    blob = sim.run_state()
    good = blob.copy()
    sim.restore_state(good)  # its own state: accepted
    with pytest.raises(fs.FsError):
        sim.restore_state(blob[:40])  # short
    bad = blob.copy()
    bad[8 * 10:8 * 10 + 4] = np.frombuffer(np.int32(7).tobytes(), np.uint8)  # ny
    with pytest.raises(fs.FsError):
        sim.restore_state(bad)
    bad = blob.copy()
    bad[-8:] = np.frombuffer(np.float64(1.5).tobytes(), np.uint8)  # accumulator
    with pytest.raises(fs.FsError):
        sim.restore_state(bad)
    sim.close()
