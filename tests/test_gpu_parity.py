"""GPU parity: the CUDA path through the C ABI against the FP64 CPU oracle on
the same seeded inputs.

FP64: the whole state is compared bit for bit (cell indices, offsets,
velocities, ids, per-cell binning, counters, every field and moment). FP32:
fields and moments within relative L2 1e-5 after one step and 1e-3 after 100
steps; integer bookkeeping exact on the GPU's own counts.
"""
import numpy as np
import pytest

from oracle import oracle as O
from tests import workloads as W

pytestmark = pytest.mark.gpu

GRIDS = [(0, O.GRID_B), (1, O.GRID_E), (2, O.GRID_BBAR), (3, O.GRID_N), (4, O.GRID_J),
         (5, O.GRID_U)]
COUNTERS = ("n_particles", "incident", "transmitted", "reflected", "escaped", "injected",
            "next_id")


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


def assert_state_equal(gpu, ref, fs, check_particles=True):
    for gw, ow in GRIDS:
        a, b = gpu.grid(gw), ref.grid(ow)
        assert a.shape == b.shape
        bad = np.argwhere(a != b)
        assert bad.size == 0, (gw, bad[:5], a[tuple(bad[0])], b[tuple(bad[0])])
    dg, dr = gpu.diag(), ref.diag()
    for k in COUNTERS:
        assert dg[k] == dr[k], (k, dg[k], dr[k])
    for k in ("kinetic", "magnetic", "px", "fs_energy", "injected_energy", "removed_energy"):
        assert dg[k] == pytest.approx(dr[k], rel=1e-12, abs=1e-12), k
    if check_particles:
        pg, pr = by_id(gpu.particles()), by_id(ref.particles())
        assert pg["id"].size == pr["id"].size
        for k in ("id", "ci", "cj", "fx", "fy", "vx", "vy", "vz"):
            bad = np.nonzero(pg[k] != pr[k])[0]
            assert bad.size == 0, (k, bad[:5], pg[k][bad[:3]], pr[k][bad[:3]])
    assert np.array_equal(gpu.grid(fs.FS_PROFILE_N), ref.grid(O.GRID_PROFILE_N))
    assert np.array_equal(gpu.grid(fs.FS_PROFILE_DB2), ref.grid(O.GRID_PROFILE_DB2))
    assert np.array_equal(gpu.histogram(), ref.histogram(-1))


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


# ---------------------------------------------------------------- FP64
def test_fp64_init_matches(fs):
    cfg = W.scaled(W.CONFIG_1D, nx=128)
    gpu = fs.FauxShock(precision=fs.FS_FP64, **cfg)
    ref = O.Oracle(**cfg)
    assert_state_equal(gpu, ref, fs)


@pytest.mark.parametrize("steps", [1, 7])
def test_fp64_1d_few_steps_bit_exact(fs, steps):
    cfg = W.scaled(W.CONFIG_1D, nx=128)
    gpu = fs.FauxShock(precision=fs.FS_FP64, **cfg)
    ref = O.Oracle(**cfg)
    gpu.step(steps)
    ref.step(steps)
    assert_state_equal(gpu, ref, fs)


def test_fp64_1d_config_full_1000_steps_bit_exact(fs):
    # the 1D FP64 configuration at full size and length
    cfg = W.CONFIG_1D
    gpu = fs.FauxShock(precision=fs.FS_FP64, **cfg)
    ref = O.Oracle(**cfg)
    for chunk in (1, 99, 400, 500):
        gpu.step(chunk)
        ref.step(chunk)
        assert_state_equal(gpu, ref, fs, check_particles=(chunk != 99))
    d = gpu.diag()
    assert d["reflected"] > 0 and d["incident"] == d["transmitted"] + d["reflected"]


@pytest.mark.parametrize("nx,n_sub", [(100, 2), (72, 3), (40, 1)])
def test_fp64_1d_ragged_field_tiles_bit_exact(fs, nx, n_sub):
    # the 1D field advance runs on 64-cell tiles with a 4 n_sub + 2 halo:
    # grids ending in a partial tile, one to three RK4 substeps per step
    cfg = W.scaled(W.CONFIG_1D, nx=nx, n_sub=n_sub)
    gpu = fs.FauxShock(precision=fs.FS_FP64, **cfg)
    ref = O.Oracle(**cfg)
    for chunk in (1, 29):
        gpu.step(chunk)
        ref.step(chunk)
        assert_state_equal(gpu, ref, fs)


@pytest.mark.parametrize("nx", [3, 8])
def test_fp64_1d_grid_smaller_than_a_field_tile_bit_exact(fs, nx):
    # the whole grid inside one 64-cell field tile and its halo: both walls
    # in the same tile
    cfg = W.scaled(W.CONFIG_1D, nx=nx, ppc=8, tile_x=min(nx, 4))
    gpu = fs.FauxShock(precision=fs.FS_FP64, **cfg)
    ref = O.Oracle(**{k: v for k, v in cfg.items() if k != "tile_x"})
    for chunk in (1, 9):
        gpu.step(chunk)
        ref.step(chunk)
        assert_state_equal(gpu, ref, fs)


@pytest.mark.parametrize("tile", [(4, 2), (8, 4), (16, 1), (2, 8)])
def test_fp64_2d_bit_exact_several_tiles(fs, tile):
    cfg = W.scaled(W.CONFIG_2D, nx=64, ny=16, ppc=8, mach_a=10.0, theta_bn_deg=20.0,
                   tile_x=tile[0], tile_y=tile[1])
    gpu = fs.FauxShock(precision=fs.FS_FP64, **cfg)
    ocfg = {k: v for k, v in cfg.items() if k not in ("tile_x", "tile_y")}
    ref = O.Oracle(**ocfg)
    gpu.step(1)
    ref.step(1)
    assert_state_equal(gpu, ref, fs)
    gpu.step(30)
    ref.step(30)
    assert_state_equal(gpu, ref, fs)


# The moment finish has the library's tile shapes compiled in for boxes more
# than a tile's accumulator high with more than three tile rows; these boxes
# sit on both sides of that rule (4x2: ny 10 compiled, 8 general; 8x4: ny 16
# compiled, 12 general), with the rows' periodic wrap in every case.
@pytest.mark.parametrize("nx,ny,tile", [(32, 10, (4, 2)), (32, 8, (4, 2)),
                                        (64, 16, (8, 4)), (64, 12, (8, 4))])
def test_fp64_2d_moment_finish_bit_exact_at_the_compiled_shape_rule(fs, nx, ny, tile):
    cfg = W.scaled(W.CONFIG_2D, nx=nx, ny=ny, ppc=8, mach_a=10.0, theta_bn_deg=20.0,
                   tile_x=tile[0], tile_y=tile[1])
    gpu = fs.FauxShock(precision=fs.FS_FP64, **cfg)
    ocfg = {k: v for k, v in cfg.items() if k not in ("tile_x", "tile_y")}
    ref = O.Oracle(**ocfg)
    for n in (1, 6):
        gpu.step(n)
        ref.step(n)
        assert_state_equal(gpu, ref, fs)


def test_fp64_2d_many_tiles_per_cta_bit_exact(fs):
    # 2x2-cell tiles on 256 x 128 cells: 8192 tiles, several per persistent CTA
    cfg = W.scaled(W.CONFIG_2D, nx=256, ny=128, ppc=8, mach_a=15.0, theta_bn_deg=10.0,
                   tile_x=2, tile_y=2)
    gpu = fs.FauxShock(precision=fs.FS_FP64, **cfg)
    assert gpu.sizes.tiles == 8192
    ocfg = {k: v for k, v in cfg.items() if k not in ("tile_x", "tile_y")}
    ref = O.Oracle(**ocfg)
    for n in (1, 9):
        gpu.step(n)
        ref.step(n)
        assert_state_equal(gpu, ref, fs)


def test_fp64_full_size_2d_workload_bit_exact(fs):
    # the FP64 2D workload at full size (4096 x 256 cells, 16 ppc, 16.8 M
    # particles) in the launch configuration the benchmark times: after one
    # and three steps every field, moment and counter equals the oracle's, and
    # a sample of particles (by id) is identical
    cfg = W.CONFIG_2D
    gpu = fs.FauxShock(precision=fs.FS_FP64, **cfg)
    ref = O.Oracle(**cfg)
    for n in (1, 2):
        gpu.step(n)
        ref.step(n)
        for gw, ow in GRIDS:
            assert np.array_equal(gpu.grid(gw), ref.grid(ow)), gw
        dg, dr = gpu.diag(), ref.diag()
        for k in COUNTERS:
            assert dg[k] == dr[k], (k, dg[k], dr[k])
    pg, pr = by_id(gpu.particles()), by_id(ref.particles())
    assert pg["id"].size == pr["id"].size
    sel = np.arange(0, pg["id"].size, 997)
    for k in ("id", "ci", "cj", "fx", "fy", "vx", "vy", "vz"):
        assert np.array_equal(pg[k][sel], pr[k][sel]), k


def test_fp32_full_size_precision_form_invariants(fs):
    # the FP32 2D precision form at full size (8192 x 512 cells, 64 ppc,
    # 268 M particles): properties that hold at any size -- exact integer
    # bookkeeping, total charge equal to the particle weight sum, finite
    # fields, and the uniform-drift equilibrium kept (E_z ~ M_A sin theta)
    cfg = W.CONFIG_2D_FP32
    gpu = fs.FauxShock(precision=fs.FS_FP32, **cfg)
    n0 = gpu.num_particles()
    assert n0 == 8192 * 512 * 64
    gpu.step(5)
    d = gpu.diag()
    assert d["status"] == 0
    assert d["n_particles"] == n0 + d["injected"] - d["transmitted"] - d["escaped"]
    assert d["incident"] == d["transmitted"] + d["reflected"]
    n = gpu.grid(fs.FS_N)
    vol = np.ones(gpu.nxn); vol[0] = vol[-1] = 0.5
    total = float((n * vol[None, :]).sum())
    assert total == pytest.approx(d["n_particles"] / 64.0, rel=2e-4)
    E = gpu.grid(fs.FS_E)
    assert np.isfinite(E).all() and np.isfinite(gpu.grid(fs.FS_B)).all()
    ez = E[:, 50:-50, 2].mean()
    assert ez == pytest.approx(30.0 * np.sin(np.radians(30.0)), rel=0.02)
    gpu.close()


def test_fp32_full_size_precision_form_error_vs_fp64(fs):
    # The FP32 precision form at full size (8192 x 512 cells, 64 ppc, 268 M
    # particles, M_A 30, theta 30 deg, seed 3) next to the same box run by
    # the plain FP64 method on the GPU, which equals the FP64 oracle bit for
    # bit (the tests above, up to the full 16.8 M-particle FP64 workload).
    # Relative L2 of every field and moment against the FP64 run: <= 1e-5
    # after one step, <= 1e-3 after 100 steps; integer bookkeeping exact in
    # each run and the injected counts equal (both draw them in FP64).
    import torch
    torch.cuda.empty_cache()
    cfg = W.CONFIG_2D_FP32
    f32 = fs.FauxShock(precision=fs.FS_FP32, **cfg)
    f64 = fs.FauxShock(precision=fs.FS_FP64, **cfg)
    n0 = 8192 * 512 * 64
    assert f32.num_particles() == n0 and f64.num_particles() == n0
    for steps, tol in ((1, 1e-5), (99, 1e-3)):
        f32.step(steps)
        f64.step(steps)
        errs = {gw: rel_l2(f32.grid(gw), f64.grid(gw)) for gw, _ in GRIDS}
        for gw, e in errs.items():
            assert e <= tol, (f32.diag()["step"], gw, errs)
        d32, d64 = f32.diag(), f64.diag()
        for d in (d32, d64):
            assert d["status"] == 0
            assert d["n_particles"] == n0 + d["injected"] - d["transmitted"] - d["escaped"]
            assert d["incident"] == d["transmitted"] + d["reflected"]
        assert d32["injected"] == d64["injected"]
        sd = 4 * np.sqrt(max(d64["reflected"], 1)) + 2
        assert abs(d32["reflected"] - d64["reflected"]) <= sd
    f32.close()
    f64.close()
    del f32, f64
    torch.cuda.empty_cache()


@pytest.mark.parametrize("chunk,ctas", [(512, 1), (512, 2)])
def test_fp64_push_launch_shapes_bit_exact(fs, chunk, ctas):
    # the launch shape is a tuning choice: FP64 results stay the oracle's
    cfg = W.scaled(W.CONFIG_2D, nx=64, ny=16, ppc=16, mach_a=10.0, theta_bn_deg=20.0)
    gpu = fs.FauxShock(precision=fs.FS_FP64, push_chunk=chunk, push_ctas_per_sm=ctas, **cfg)
    ref = O.Oracle(**cfg)
    gpu.step(12)
    ref.step(12)
    assert_state_equal(gpu, ref, fs)


@pytest.mark.parametrize("chunk,ctas", [(512, 0), (576, 2), (512, 2)])
def test_fp32_push_launch_shapes_within_tolerance(fs, chunk, ctas):
    cfg = W.scaled(W.CONFIG_2D_FP32, nx=64, ny=16)
    gpu = fs.FauxShock(precision=fs.FS_FP32, push_chunk=chunk, push_ctas_per_sm=ctas, **cfg)
    ref = O.Oracle(**cfg)
    gpu.step(20)
    ref.step(20)
    for gw, ow in GRIDS:
        assert rel_l2(gpu.grid(gw), ref.grid(ow)) <= 1e-3, gw
    d = gpu.diag()
    assert d["status"] == 0 and d["injected"] == ref.diag()["injected"]


def test_fp64_multi_chunk_tiles_bit_exact(fs):
    # 128 cells x 32 ppc = 4096 particles per tile: several shared-memory chunks
    cfg = W.scaled(W.CONFIG_1D, nx=256, tile_x=128)
    gpu = fs.FauxShock(precision=fs.FS_FP64, **cfg)
    ocfg = {k: v for k, v in cfg.items() if k != "tile_x"}
    ref = O.Oracle(**ocfg)
    gpu.step(20)
    ref.step(20)
    assert_state_equal(gpu, ref, fs)


def test_fp64_cosmic_ray_source_and_open_thermal(fs):
    # the paper's set-up: thermal plasma open at the faux shock, a cosmic-ray
    # species injected at the faux shock that passes or returns (Sec. 2)
    cfg = W.scaled(W.CONFIG_1D, nx=128, fs_mode_thermal=O.FS_OPEN, cr_enable=1,
                   p_iso=40.0, n_cr_ratio=0.01)
    gpu = fs.FauxShock(precision=fs.FS_FP64, **cfg)
    ref = O.Oracle(**cfg)
    gpu.step(150)
    ref.step(150)
    assert_state_equal(gpu, ref, fs)
    assert gpu.histogram(cr_only=True).sum() > 0
    assert np.array_equal(gpu.histogram(cr_only=True), ref.histogram(1))
    # cosmic rays stream away from the wall (no turbulence yet to return them)
    p = gpu.particles()
    ncr = int(((p["id"] & fs.ID_CR) != 0).sum())
    d = gpu.diag()
    assert ncr > 0 and d["injected"] >= 2 * ncr


def test_fp64_direct_launches_equal_graph_replay(fs):
    # fs_step replays a captured CUDA graph after its first step; with
    # use_graph = 0 every step launches directly: both equal the oracle
    cfg = W.scaled(W.CONFIG_1D, nx=128)
    direct = fs.FauxShock(precision=fs.FS_FP64, use_graph=0, **cfg)
    ref = O.Oracle(**cfg)
    direct.step(40)
    ref.step(40)
    assert_state_equal(direct, ref, fs)


def test_fp64_downstream_frame_return(fs):
    cfg = W.scaled(W.CONFIG_1D, nx=64, fs_speed_frame=O.FRAME_DOWNSTREAM, r_comp=3.0)
    gpu = fs.FauxShock(precision=fs.FS_FP64, **cfg)
    ref = O.Oracle(**cfg)
    gpu.step(60)
    ref.step(60)
    assert_state_equal(gpu, ref, fs)


def test_fp64_periodic_cold_wave_bit_exact(fs):
    # periodic box, quiet start, seeded circularly polarised mode
    nx, ppc, k = 64, 8, 2 * np.pi / 32.0
    cfg = dict(dim=1, nx=nx, dx=0.5, dt=0.01, ppc=ppc, init_plasma=0, bc_x=O.BC_PERIODIC,
               mach_a=0.0, beta_i=0.0, beta_e=0.5)
    gpu = fs.FauxShock(precision=fs.FS_FP64, **cfg)
    ref = O.Oracle(**cfg)
    xc = (np.arange(nx) + 0.5) * 0.5
    B = ref.grid(O.GRID_B)
    B[0, :, 1] = 1e-2 * np.cos(k * xc)
    B[0, :, 2] = 1e-2 * np.sin(k * xc)
    load = W.quiet_load(nx, 1, ppc, vel=lambda x, y: np.stack(
        [0.01 * np.sin(0.5 * k * x), 0.02 * np.cos(k * x * 0.5), 0 * x]))
    for sim in (gpu, ref):
        sim.load_fields(B) if sim is gpu else sim.set_B(B)
        sim.inject(*load)
    gpu.step(50)
    ref.step(50)
    assert_state_equal(gpu, ref, fs)


def test_fp64_periodic_2d_bell_current_bit_exact(fs):
    cfg = dict(dim=2, nx=32, ny=8, dx=0.5, dy=0.5, dt=0.01, ppc=4, bc_x=O.BC_PERIODIC,
               mach_a=1.0, beta_i=0.5, beta_e=0.5, j_cr_ext=0.2, seed=9)
    gpu = fs.FauxShock(precision=fs.FS_FP64, **cfg)
    ref = O.Oracle(**cfg)
    gpu.step(40)
    ref.step(40)
    assert_state_equal(gpu, ref, fs)


def test_fp64_fast_particles_far_movers(fs):
    # particles that cross several cells (and tiles) in one step take the
    # far-mover path; results must not change
    cfg = dict(dim=1, nx=128, dx=0.5, dt=0.01, ppc=32, init_plasma=0, bc_x=O.BC_PERIODIC,
               mach_a=0.0, beta_i=0.0, beta_e=0.5, tile_x=8)
    gpu = fs.FauxShock(precision=fs.FS_FP64, **cfg)
    ocfg = {k: v for k, v in cfg.items() if k != "tile_x"}
    ref = O.Oracle(**ocfg)
    rng = np.random.default_rng(5)
    load = W.random_particles(rng, 3000, 128, 1, vscale=150.0)
    gpu.inject(*load)
    ref.inject(*load)
    for _ in range(3):
        gpu.step(5)
        ref.step(5)
        assert_state_equal(gpu, ref, fs)


def test_fp64_empty_box_and_offsets_at_edges(fs):
    cfg = dict(dim=2, nx=16, ny=8, dx=0.5, dy=0.5, dt=0.005, ppc=4, init_plasma=0,
               mach_a=5.0, inject_thermal=0)
    gpu = fs.FauxShock(precision=fs.FS_FP64, **cfg)
    ref = O.Oracle(**cfg)
    gpu.step(3)
    ref.step(3)
    assert gpu.num_particles() == 0
    assert_state_equal(gpu, ref, fs)
    # particles sitting on cell edges and just below 1, moving both ways
    ci = np.array([0, 0, 15, 15, 7, 3], np.int32)
    cj = np.array([0, 7, 0, 7, 4, 2], np.int32)
    fx = np.array([0.0, 1 - 2**-53, 0.0, 1 - 2**-53, 0.5, 0.0])
    fy = np.array([0.0, 1 - 2**-53, 1 - 2**-53, 0.0, 0.5, 0.25])
    vx = np.array([-30.0, 30.0, -1e-9, 1e-9, 0.0, -200.0])
    vy = np.array([-5.0, 5.0, 1e-17, -1e-17, 0.0, 77.0])
    vz = np.zeros(6)
    gpu.inject(ci, cj, fx, fy, vx, vy, vz)
    ref.inject(ci, cj, fx, fy, vx, vy, vz)
    for _ in range(4):
        gpu.step(1)
        ref.step(1)
        assert_state_equal(gpu, ref, fs)


def test_capacity_overflow_is_reported_not_faulted(fs):
    cfg = dict(dim=1, nx=32, ppc=2, capacity_factor=1.0, init_plasma=0, mach_a=0.0,
               inject_thermal=0, tile_x=16)
    gpu = fs.FauxShock(precision=fs.FS_FP64, **cfg)
    cap = gpu.sizes.particle_capacity
    n = int(cap) + 100
    ci = np.zeros(n, np.int32)
    with pytest.raises(fs.FsError) as e:
        gpu.inject(ci, ci, np.full(n, 0.5), np.zeros(n), np.zeros(n), np.zeros(n), np.zeros(n))
    assert e.value.code == -2
    # the handle keeps reporting the sticky error
    with pytest.raises(fs.FsError):
        gpu.diag()


def test_inject_rejects_out_of_range(fs):
    gpu = fs.FauxShock(precision=fs.FS_FP64, dim=1, nx=32, ppc=2)
    for bad in (dict(ci=[32]), dict(ci=[-1]), dict(fx=[1.0]), dict(fx=[-0.1]),
                dict(vx=[np.nan])):
        a = dict(ci=[3], cj=[0], fx=[0.5], fy=[0.0], vx=[0.0], vy=[0.0], vz=[0.0])
        a.update(bad)
        with pytest.raises(fs.FsError) as e:
            gpu.inject(**{k: np.array(v) for k, v in a.items()})
        assert e.value.code == -1


def test_inject_large_rejects_a_bad_value_and_inserts_nothing(fs):
    # inputs over a million particles are checked on several host threads;
    # one bad value deep inside fails the call before anything is inserted
    gpu = fs.FauxShock(precision=fs.FS_FP64, dim=2, nx=256, ny=64, ppc=64, init_plasma=0,
                       inject_thermal=0, capacity_factor=2.0)
    rng = np.random.default_rng(9)
    n = 1_200_000
    a = dict(ci=rng.integers(0, 256, n).astype(np.int32),
             cj=rng.integers(0, 64, n).astype(np.int32), fx=rng.uniform(0, 1, n),
             fy=rng.uniform(0, 1, n), vx=rng.normal(0, 1, n), vy=rng.normal(0, 1, n),
             vz=rng.normal(0, 1, n))
    for key, val in (("fy", 1.0), ("cj", 64), ("vz", np.inf)):
        b = {k: v.copy() for k, v in a.items()}
        b[key][987_654] = val
        with pytest.raises(fs.FsError) as e:
            gpu.inject(**b)
        assert e.value.code == -1
        assert gpu.num_particles() == 0
    gpu.inject(**a)
    assert gpu.num_particles() == n
    gpu.close()


@pytest.mark.parametrize("prec,with_ids", [("fp64", False), ("fp64", True), ("fp32", False)])
def test_inject_round_trip(fs, prec, with_ids):
    # FP64 without ids: columns copied as they are, cell and ids formed on the
    # device; with ids, and FP32: packed on the host. Every particle comes
    # back with its cell, offsets, velocity and id (ids in input order when
    # the library assigns them).
    precision = fs.FS_FP64 if prec == "fp64" else fs.FS_FP32
    gpu = fs.FauxShock(precision=precision, dim=2, nx=64, ny=32, ppc=64, init_plasma=0,
                       inject_thermal=0, capacity_factor=2.0)
    rng = np.random.default_rng(11)
    n = 200_000
    a = dict(ci=rng.integers(0, 64, n).astype(np.int32),
             cj=rng.integers(0, 32, n).astype(np.int32), fx=rng.uniform(0, 1, n),
             fy=rng.uniform(0, 1, n), vx=rng.normal(0, 1, n), vy=rng.normal(0, 1, n),
             vz=rng.normal(0, 1, n))
    ids = rng.permutation(n).astype(np.uint32) + 5 if with_ids else None
    gpu.inject(**a, ids=ids)
    p = gpu.particles()
    assert len(p["id"]) == n
    want = ids if with_ids else np.arange(n, dtype=np.uint32)
    order = np.argsort(p["id"])
    src = np.argsort(want)
    assert np.array_equal(p["id"][order], want[src])
    for k in ("ci", "cj"):
        assert np.array_equal(p[k][order], a[k][src]), k
    cast = (lambda x: x) if prec == "fp64" else (lambda x: x.astype(np.float32).astype(np.float64))
    for k in ("fx", "fy", "vx", "vy", "vz"):
        got, exp = p[k][order], cast(a[k][src])
        if k in ("fx", "fy") and prec == "fp32":
            exp = np.minimum(exp, np.float64(np.nextafter(np.float32(1), np.float32(0))))
        assert np.array_equal(got, exp), k
    # the next ids continue after the largest one in use
    d = gpu.diag()
    assert d["next_id"] == (int(want.max()) + 1)
    gpu.close()


# ---------------------------------------------------------------- FP32
@pytest.mark.parametrize("dim", [1, 2, "2-ragged", "2-tiny", "2-odd", "2-interior"])
def test_fp32_fields_within_tolerance(fs, dim):
    if dim == 1:
        cfg = W.scaled(W.CONFIG_1D, nx=256)
    elif dim == 2:
        cfg = W.scaled(W.CONFIG_2D_FP32, nx=64, ny=16, ppc=16)
    elif dim == "2-interior":
        # a whole number of 32 x 16-cell field tiles, four columns: the two
        # interior columns take the launch with the tile sizes compiled in
        cfg = W.scaled(W.CONFIG_2D_FP32, nx=128, ny=32, ppc=16)
    elif dim == "2-tiny":
        # the whole box in one 32 x 16-cell field tile, rows repeated by the
        # periodic halo
        cfg = W.scaled(W.CONFIG_2D_FP32, nx=5, ny=3, ppc=16)
    elif dim == "2-odd":
        cfg = W.scaled(W.CONFIG_2D_FP32, nx=33, ny=17, ppc=16, tile_x=3, tile_y=1)
    else:
        # the 2D field advance runs on 32 x 16-cell tiles: partial tiles in
        # x and y, three substeps (halo 4, then 5 in the last)
        cfg = W.scaled(W.CONFIG_2D_FP32, nx=72, ny=20, ppc=16, n_sub=3)
    gpu = fs.FauxShock(precision=fs.FS_FP32, **cfg)
    ref = O.Oracle(**{k: v for k, v in cfg.items() if k not in ("tile_x", "tile_y")})
    gpu.step(1)
    ref.step(1)
    for gw, ow in GRIDS:
        assert rel_l2(gpu.grid(gw), ref.grid(ow)) <= 1e-5, gw
    gpu.step(99)
    ref.step(99)
    errs = {gw: rel_l2(gpu.grid(gw), ref.grid(ow)) for gw, ow in GRIDS}
    for gw, e in errs.items():
        assert e <= 1e-3, (gw, errs)
    d = gpu.diag()
    n0 = cfg["nx"] * cfg["ny"] * cfg["ppc"]
    assert d["n_particles"] == n0 + d["injected"] - d["transmitted"] - d["escaped"]
    assert d["incident"] == d["transmitted"] + d["reflected"]
    dr = ref.diag()
    assert d["injected"] == dr["injected"]
    sd = 4 * np.sqrt(max(dr["reflected"], 1)) + 2
    assert abs(d["reflected"] - dr["reflected"]) <= sd


def test_field_stability_number_and_unstable_report(fs):
    # z = h [(4/dx^2 (+4/dy^2)) |Bbar| / n + (2/dx (+2/dy)) |u|], maximum over
    # nodes, from the run's own node fields; FS_EUNSTABLE above 2 sqrt 2
    for dim, dx, dt, unstable in ((1, 0.5, 0.005, False), (2, 0.5, 0.0025, False),
                                  (1, 0.05, 0.02, True)):
        p = W.scaled(W.CONFIG_1D if dim == 1 else W.CONFIG_2D, nx=64,
                     ny=1 if dim == 1 else 16, dx=dx, dy=dx, dt=dt, ppc=8)
        sim = fs.FauxShock(precision=fs.FS_FP64, **p)
        d = sim.diag()
        bb, n, u = sim.grid(fs.FS_BBAR), sim.grid(fs.FS_N), sim.grid(fs.FS_U)
        kk = 4 / dx**2 * (2 if dim == 2 else 1)
        ka = 2 / dx * (2 if dim == 2 else 1)
        z = dt / 2 * (kk * np.linalg.norm(bb, axis=-1) / n + ka * np.linalg.norm(u, axis=-1))
        assert d["max_z"] == pytest.approx(z.max(), rel=1e-12)
        assert d["unstable"] == unstable
        assert (d["max_z"] > fs.FS_RK4_Z_MAX) == unstable
        sim.close()


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_tile_buckets_stay_cell_sorted(fs, prec):
    # Each tile's bucket (exported contiguously, in bucket order) is sorted by
    # cell up to a tail of particles appended since the push: those moved in
    # from other tiles and the injected ones (a few per cent per step).
    p = W.scaled(W.CONFIG_2D_FP32, nx=256, ny=64, seed=5)
    sim = fs.FauxShock(precision=fs.FS_FP64 if prec == "fp64" else fs.FS_FP32, **p)
    tx, ty = sim.sizes.tile_x, sim.sizes.tile_y
    for steps in (1, 4):
        sim.step(steps)
        q = sim.particles()
        i, j = q["ci"], q["cj"]
        tile = (j // ty) * (p["nx"] // tx) + i // tx
        local = (j % ty) * tx + i % tx
        sorted_n, k, n = 0, 0, len(tile)
        while k < n:
            e = k + 1
            while e < n and tile[e] == tile[k]:
                e += 1
            run = local[k:e]
            desc = np.nonzero(np.diff(run) < 0)[0]
            sorted_n += (desc[0] + 1) if desc.size else (e - k)
            k = e
        assert sorted_n >= 0.9 * n, (steps, sorted_n / n)
    assert sim.diag()["status"] == 0
    sim.close()


@pytest.mark.parametrize("mode", ["shock", "open+cr"])
def test_fp32_2d_precision_form_tiles_within_tolerance(fs, mode):
    # the precision form's shape: 64 ppc in 4 x 2-cell tiles (512 particles,
    # the tile push's FP32 chunk), returning or open faux shock
    cfg = W.scaled(W.CONFIG_2D_FP32, nx=64, ny=16)
    if mode == "open+cr":
        cfg.update(fs_mode_thermal=O.FS_OPEN, cr_enable=1)
    gpu = fs.FauxShock(precision=fs.FS_FP32, **cfg)
    assert (gpu.sizes.tile_x, gpu.sizes.tile_y) == (4, 2)
    ref = O.Oracle(**cfg)
    gpu.step(1)
    ref.step(1)
    for gw, ow in GRIDS:
        assert rel_l2(gpu.grid(gw), ref.grid(ow)) <= 1e-5, (gw, mode)
    gpu.step(99)
    ref.step(99)
    errs = {gw: rel_l2(gpu.grid(gw), ref.grid(ow)) for gw, ow in GRIDS}
    assert max(errs.values()) <= 1e-3, errs
    d, dr = gpu.diag(), ref.diag()
    assert d["status"] == 0
    assert d["injected"] == dr["injected"]
    assert d["incident"] == d["transmitted"] + d["reflected"]
    n0 = cfg["nx"] * cfg["ny"] * cfg["ppc"]
    assert d["n_particles"] == n0 + d["injected"] - d["transmitted"] - d["escaped"]
    sd = 4 * np.sqrt(max(dr["reflected"], 1)) + 2
    assert abs(d["reflected"] - dr["reflected"]) <= sd
    gpu.close()


def test_fp64_fma_rate_is_plausible(fs):
    # the FP64 roofline denominator: near GB300's nominal 0.625 T FMA/s
    r = fs.fp64_fma_rate(1 << 12)
    assert 0.2e12 < r < 1.0e12, r
