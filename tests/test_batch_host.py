"""Host logic of batched ensembles (no GPU): the CTA-group planner behind
fs_batch_plan, the configuration-4 parameter draws and the tile autotuner's
shape rule."""
import numpy as np
import pytest

from tests import workloads as W


@pytest.fixture(scope="module")
def fs():
    from paper_2507_14282_gb300 import build
    build.build()
    from paper_2507_14282_gb300 import fs as m
    return m


def check_plan(n, t, cmax, out):
    out = np.asarray(out)
    assert len(out) == len(n)
    assert out.min() >= 1
    assert np.all(out <= np.asarray(t))
    assert out.sum() <= cmax
    return out


def test_plan_is_proportional_and_fills_the_gpu(fs):
    rng = np.random.default_rng(7)
    n = rng.integers(10_000, 2_000_000, size=64)
    t = n // 256 + 1
    cmax = 456
    out = check_plan(n, t, cmax, fs.batch_plan(n, t, cmax))
    assert out.sum() == cmax  # every run can take more CTAs than it gets
    load = n / out
    # integer groups: particles per CTA stay close to even
    assert load.max() / load.mean() < 1.6
    # no CTA moved from the lightest-loaded group to the heaviest would help
    i, j = np.argmax(load), np.argmin(np.where(out > 1, n / np.maximum(out - 1, 1), np.inf))
    assert n[i] / (out[i] + 1) < n[j] / (out[j] - 1) or out[j] == 1


def test_plan_caps_groups_at_tile_counts(fs):
    n = [1_000_000, 10, 10]
    t = [4, 1, 1]
    out = check_plan(n, t, 100, fs.batch_plan(n, t, 100))
    assert list(out) == [4, 1, 1]  # the big run cannot use more CTAs than tiles


def test_plan_exact_small_cases(fs):
    assert fs.batch_plan([100, 100], [50, 50], 10) == [5, 5]
    assert fs.batch_plan([300, 100], [50, 50], 8) == [6, 2]
    assert fs.batch_plan([0, 0, 0], [5, 5, 5], 3) == [1, 1, 1]
    # a tiny run keeps one CTA even when proportion says zero
    assert fs.batch_plan([1_000_000, 1], [100, 100], 10) == [9, 1]


@pytest.mark.parametrize("args", [
    ([1, 2, 3], [1, 1, 1], 2),      # more runs than CTAs
    ([1, -2], [1, 1], 8),           # negative count
    ([1, 2], [1, 0], 8),            # empty tile range
])
def test_plan_rejects(fs, args):
    with pytest.raises(fs.FsError):
        fs.batch_plan(*args)


def test_config4_draws_are_seeded_and_in_range():
    a = W.config4_runs()
    b = W.config4_runs()
    assert a == b and len(a) == 64
    assert [r["seed"] for r in a] == list(range(100, 164))
    for r in a:
        assert 512 <= r["nx"] <= 8192 and r["nx"] % 32 == 0
        assert r["ppc"] in (32, 64, 128, 256)
        assert 5.0 <= r["mach_a"] <= 100.0
        assert 0.0 <= r["theta_bn_deg"] <= 60.0
        assert r["beta_i"] == r["beta_e"] and r["beta_i"] in (0.5, 1.0, 2.0)
        assert r["dt"] == pytest.approx(min(0.005, 0.05 / r["mach_a"]))
        assert r["dt"] * r["mach_a"] / r["dx"] <= 0.1 + 1e-12  # at most 0.1 cell/step drift
    # log-uniform lengths: both ends of the range occur
    nx = np.array([r["nx"] for r in a])
    assert nx.min() < 1024 and nx.max() > 4096
    assert len({r["ppc"] for r in a}) == 4


def test_tile_rule():
    from paper_2507_14282_gb300 import tune
    assert tune.divisors(12) == [2, 3, 4, 6, 12]
    assert tune.tile_for(2048, 64, 512) == 8
    assert tune.tile_for(2048, 256, 512) == 2
    assert tune.tile_for(5792, 128, 512) == 4   # 5792 = 2^5 * 181
    assert tune.tile_for(5792, 32, 1024) == 32


def test_tuner_2d_candidates_and_launch_shapes():
    from paper_2507_14282_gb300 import tune, fs
    c = tune.tile_candidates_2d(1024, 64, 64)
    assert (4, 2) in c and (8, 1) in c and (2, 4) in c
    for tx, ty in c:
        assert 1024 % tx == 0 and 64 % ty == 0 and tx >= 2
        assert 128 <= tx * ty * 64 <= 1024
    counts = [tx * ty for tx, ty in c]
    assert counts == sorted(counts)
    # a box whose sides admit no shape in range gives none
    assert tune.tile_candidates_2d(7, 1, 1000) == []
    assert (0, 0) in tune.launch_shapes(fs.FS_FP32) and (576, 0) in tune.launch_shapes(fs.FS_FP32)
    assert all(c in (0, 512) for c, _ in tune.launch_shapes(fs.FS_FP64))


def test_tuner_limits_batch_runs_to_compiled_widths():
    from paper_2507_14282_gb300 import tune, fs
    w = fs.FsBatch.COMPILED_WIDTHS
    # 32 ppc on 4096 cells: targets 128 / 256 / 512 give widths 4 / 8 / 16,
    # 1024 gives 32, which no batched push has compiled in
    assert tune.targets_1d(4096, 32, None) == list(tune.TARGETS)
    assert tune.targets_1d(4096, 32, w) == [128, 256, 512]
    assert tune.targets_1d(4096, 256, w) == [1024]
    for t in tune.targets_1d(4096, 64, w):
        assert tune.tile_for(4096, 64, t) in w
    # no candidate within the widths: all of them
    assert tune.targets_1d(4099, 64, w) == list(tune.TARGETS)
    a, b = tune.Autotuner(), tune.Autotuner(widths=w)
    assert a.key(1, 32, fs.FS_FP32) == "dim1-ppc32-fp32"
    assert b.key(1, 32, fs.FS_FP32) == "dim1-ppc32-fp32-w4.8.16"
    assert b.key(2, 64, fs.FS_FP32) == a.key(2, 64, fs.FS_FP32)
