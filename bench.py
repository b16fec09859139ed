"""Benchmark: particle-steps/s of the full faux-shock hybrid step on GB300.

Default workload (N=1): the 2D production-shaped faux-shock box computed in
FP64 (4096 x 256 cells, dx = 0.5 d_i, 16 ppc = 16.8 M particles, M_A = 20,
theta_Bn = 0, beta_i = beta_e = 1, dt = 0.0025, seed 2). The same run also
times the FP32 precision form (8192 x 512 cells, 64 ppc = 268 M particles,
M_A = 30, theta_Bn = 30 deg, dt = 0.002, seed 3) and reports it under "fp32"
(the metric compares FP32 with FP64), and the batched ensemble of 64 uneven
1D FP32 runs stepped together (reported under "ensemble", with the same runs
stepped one after another beside it).

A step is one full hybrid step: gather, Boris push, faux-shock pass/return,
cell binning, moment deposition, moment finish, Ohm's law + Faraday RK4
substeps and the node packing for the next gather. Inputs (particle state,
1.6 GB FP64 / 15 GB FP32) are larger than L2 (129 MB), so no L2 flush is
needed between steps.

Multi-GPU: the path does not shard (one box per GPU); N > 1 runs N
independent replicas (weak scaling), one per rank.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "particle-steps/s on 1 GB300 (full hybrid step), % HBM roofline; FP32 vs FP64"
UNIT = "particle-steps/s"

FP64_WORKLOAD = dict(dim=2, nx=4096, ny=256, dx=0.5, dy=0.5, dt=0.0025, mach_a=20.0,
                     theta_bn_deg=0.0, beta_i=1.0, beta_e=1.0, ppc=16, seed=2)
FP32_WORKLOAD = dict(dim=2, nx=8192, ny=512, dx=0.5, dy=0.5, dt=0.002, mach_a=30.0,
                     theta_bn_deg=30.0, beta_i=1.0, beta_e=1.0, ppc=64, seed=3)
WORKLOAD_NAME = ("2D faux-shock hybrid PIC, 4096x256 cells, dx=0.5 d_i, 16 ppc "
                 "(16.8M protons), M_A=20, theta_Bn=0, beta_i=beta_e=1, dt=0.0025, "
                 "FP64 plain method, seed 2")
FP32_NAME = ("2D faux-shock hybrid PIC precision form, 8192x512 cells, 64 ppc "
             "(268M protons), M_A=30, theta_Bn=30 deg, beta=1, dt=0.002, FP32, seed 3")

ENSEMBLE_NAME = ("batched ensemble: 64 independent 1D faux-shock runs in FP32, N_x "
                 "log-uniform in 512..8192, ppc in {32,64,128,256}, M_A 5..100, theta_Bn "
                 "0..60 deg, beta in {0.5,1,2}, dt = min(0.005, 0.1 dx/M_A), seeds 100..163 "
                 "(Philox), autotuned tiles; one graph-captured batched step")

# Algorithmic bytes of the particle push per particle-step: the particle state
# (int32 cell, offsets, velocity, uint32 id) read once and written once.
def particle_bytes(prec_bytes: int, dim: int) -> int:
    return 2 * (4 + prec_bytes * dim + 3 * prec_bytes + 4)


# Grid traffic per cell per step on a single pass (moments write + read 8
# words, B read + write 6, E write 3, E + Bbar read by the gather 6).
GRID_WORDS_PER_CELL = 23
# FP64-pipe operations of the FP64 push per particle-step in 2D, from ncu
# (sm__thread_inst_executed_pipe_fp64_pred_on.sum over the particles of one
# launch of the 1024 x 256-cell case: 408.2 M / 4 194 771; DADD + DMUL + DFMA
# alone give 96.9); an FMA is one pipe operation, like the denominator.
FP64_OPS_PER_PARTICLE_STEP = 97.3
FP64_OPS_SOURCE = ("ncu sm__thread_inst_executed_pipe_fp64_pred_on.sum / particles, "
                   "1024x256-cell case of the FP64 workload")
PHASE_TIMING = ("value: the product path (graph replay, no phase events); phases and "
                "kernel_ms: a second pass of the same run with per-phase CUDA events "
                "(steps launched directly)")
# FP64 throughput of GB300: 1.25 TFLOP/s nominal counts an FMA as two; the
# scheme issues unfused adds and multiplies, one operation per pipe slot.
# The roofline takes the rate measured on the GPU (fs_fp64_fma_rate), this
# nominal figure only if the measurement fails.
FP64_PEAK_OPS = 0.625e12


# DRAM bytes per particle of one k_push launch, from ncu (dram__bytes_read.sum
# + dram__bytes_write.sum) on a 1024 x 256-cell case of the same kernel, scaled
# by the particles of a launch; valid only while the kernel sources are the
# ones the counters were taken on (their hash below), else reported as null.
PUSH_TRAFFIC = {"fp32": (506.448128e6 + 448.124416e6) / 16779950,
                "fp64": (224.050944e6 + 175.183872e6) / 4194771}
PUSH_SOURCES = ("paper_2507_14282_gb300/csrc/fs_push.cuh",
                "paper_2507_14282_gb300/csrc/fs_engine.cuh")
# hash of PUSH_SOURCES when each precision's counters were taken
PUSH_SOURCES_SHA1 = {"fp32": "f2d64bea1b9ff0cea678960c8fe9e907546835bf",
                     "fp64": "f2d64bea1b9ff0cea678960c8fe9e907546835bf"}


def push_sources_sha1() -> str:
    import hashlib
    h = hashlib.sha1()
    for f in PUSH_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def traffic_per_launch(prec: str, n: float):
    if push_sources_sha1() != PUSH_SOURCES_SHA1[prec]:
        return None
    return PUSH_TRAFFIC[prec] * n


def load_peaks() -> dict:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for n, v in zip(names, parts[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        busy = [s for s in sm if s > 0.5 * max(sm)] or sm
        return {"sm_mhz": statistics.median(busy), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup(n_gpus: int, backend: str = "nccl"):
    if n_gpus <= 1 or "RANK" not in os.environ:
        return 0, 1, 0, None
    import torch.distributed as dist
    dist.init_process_group(backend)
    return (dist.get_rank(), dist.get_world_size(), int(os.environ.get("LOCAL_RANK", 0)),
            dist)


def replica_value(n_mean: float, steps: int, ms_local: float, dist, device="cpu"):
    """Whole-job throughput of independent replicas (one box per rank): the
    particles every rank pushed per step, summed, times the steps, over the
    slowest rank's time. Returns (value, ms of the slowest rank)."""
    import torch
    if not dist:
        return n_mean * steps / (ms_local * 1e-3), ms_local
    t = torch.tensor([ms_local], dtype=torch.float64, device=device)
    n = torch.tensor([n_mean], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(n, op=dist.ReduceOp.SUM)
    return float(n.item()) * steps / (float(t.item()) * 1e-3), float(t.item())


def timed_run(fs, torch, params: dict, prec, steps: int, warmup: int, dist, device,
              sample_clocks: bool, local_rank: int, prof_steps: int):
    """Device-resident timing of `steps` steps on the product path (fs_step
    replaying its captured CUDA graph, no per-phase events), then a second,
    profiled pass of `prof_steps` steps whose per-phase CUDA events (recorded
    by the library on its stream; the steps launch directly) give the phase
    and dominant-kernel durations. Returns measurements."""
    sim = fs.FauxShock(device=device, precision=prec, **params)
    stream = sim.stream
    sim.step(warmup)
    torch.cuda.synchronize()
    n0 = sim.num_particles()
    l0 = sim.diag()["launches"]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clk = ClockSampler(local_rank) if sample_clocks else None
    if clk:
        clk.start()
        time.sleep(0.3)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        sim.step(1)
    e1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = clk.stop() if clk else None
    ms = e0.elapsed_time(e1)
    d = sim.diag()
    n1 = d["n_particles"]
    launches = d["launches"] - l0
    # second pass: per-phase events, the fused particle step among them
    sim.profile(True)
    sim.profile_read()
    e0.record(stream)
    for _ in range(prof_steps):
        sim.step(1)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_prof = e0.elapsed_time(e1)
    phases = sim.profile_read()
    sim.profile(False)
    n2 = sim.num_particles()
    sizes = sim.sizes
    out = dict(ms_total=ms, n_mean=0.5 * (n0 + n1), launches=launches, clocks=clocks,
               sim=sim, tiles=sizes.tiles, tile=(sizes.tile_x, sizes.tile_y),
               phases={k: v[0] / max(v[1], 1) for k, v in phases.items()},
               prof_ms_per_step=ms_prof / max(prof_steps, 1), prof_steps=prof_steps,
               prof_n_mean=0.5 * (n1 + n2))
    return out


def ours(args):
    import torch
    from paper_2507_14282_gb300 import fs

    rank, world, local_rank, dist = dist_setup(args.gpus)
    torch.cuda.set_device(local_rank)
    device = f"cuda:{local_rank}"
    peaks = load_peaks()
    hbm = peaks.get("hbm_gbs")
    peak_src = "measured" if hbm else "fallback"
    hbm = hbm or 6800.0

    try:  # the FP64 FMA rate of this GPU, best of three
        fp64_peak = max(fs.fp64_fma_rate() for _ in range(3))
        fp64_src = "measured (FP64 FMA microbenchmark, fs_fp64_fma_rate)"
    except Exception:
        fp64_peak = FP64_PEAK_OPS
        fp64_src = "derived from nominal FP64 1.25 TFLOP/s (FMA=2)"
    res64 = timed_run(fs, torch, FP64_WORKLOAD, fs.FS_FP64, args.steps, args.warmup, dist,
                      device, True, local_rank, args.prof_steps)
    value, t64 = replica_value(res64["n_mean"], args.steps, res64["ms_total"], dist, device)
    ms_step = t64 / args.steps
    pb64 = particle_bytes(8, 2)
    grid_b64 = GRID_WORDS_PER_CELL * 8 / FP64_WORKLOAD["ppc"]
    step_bw64 = res64["n_mean"] * (pb64 + grid_b64) / (ms_step * 1e-3) / 1e9
    kern64 = res64["phases"]["push"]
    achieved_ops = res64["prof_n_mean"] * FP64_OPS_PER_PARTICLE_STEP / (kern64 * 1e-3) / 1e12
    roofline = {"bound": "alu", "kernel": "k_push<double,2>",
                "achieved": achieved_ops, "peak": fp64_peak / 1e12,
                "unit": "TFLOP/s (FP64 ops)",
                "frac": achieved_ops / (fp64_peak / 1e12),
                "peak_nominal": FP64_PEAK_OPS / 1e12,
                "traffic": traffic_per_launch("fp64", res64["n_mean"]),
                "traffic_unit": "bytes per launch",
                "kernel_ms": kern64,
                "ops_per_particle_step": FP64_OPS_PER_PARTICLE_STEP,
                "ops_source": FP64_OPS_SOURCE,
                "hbm_achieved_gbs": res64["prof_n_mean"] * pb64 / (kern64 * 1e-3) / 1e9,
                "hbm_peak_gbs": hbm,
                "hbm_frac": res64["prof_n_mean"] * pb64 / (kern64 * 1e-3) / 1e9 / hbm,
                "peak_source": fp64_src,
                "step_hbm_frac": step_bw64 / hbm,
                "phases_ms": res64["phases"],
                "timing": PHASE_TIMING,
                "profiled_ms_per_step": res64["prof_ms_per_step"]}
    gpu_launches = res64["launches"]
    res64["sim"].close()
    del res64["sim"]
    torch.cuda.empty_cache()

    fp32 = None
    if not args.skip_fp32:
        res32 = timed_run(fs, torch, FP32_WORKLOAD, fs.FS_FP32, args.steps32, args.warmup,
                          dist, device, False, local_rank, args.prof_steps)
        v32, t32 = replica_value(res32["n_mean"], args.steps32, res32["ms_total"], dist, device)
        ms32 = t32 / args.steps32
        pb32 = particle_bytes(4, 2)
        gb32 = GRID_WORDS_PER_CELL * 4 / FP32_WORKLOAD["ppc"]
        kern32 = res32["phases"]["push"]
        ach = res32["prof_n_mean"] * pb32 / (kern32 * 1e-3) / 1e9
        fp32 = {"workload": FP32_NAME, "value": v32, "unit": UNIT, "ms_per_step": ms32,
                "steps": args.steps32, "n_particles": res32["n_mean"],
                "bytes_per_particle_step": pb32 + gb32,
                "step_roofline_frac": res32["n_mean"] * (pb32 + gb32) / (ms32 * 1e-3) / 1e9 / hbm,
                "roofline": {"bound": "hbm", "kernel": "k_push<float,2>", "achieved": ach,
                             "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                             "traffic": traffic_per_launch("fp32", res32["n_mean"]),
                             "traffic_unit": "bytes per launch",
                             "kernel_ms": kern32, "peak_source": peak_src},
                "phases_ms": res32["phases"], "timing": PHASE_TIMING,
                "profiled_ms_per_step": res32["prof_ms_per_step"],
                "vs_fp64": v32 / value, "gpu_launches": res32["launches"]}
        gpu_launches += res32["launches"]
        res32["sim"].close()
        del res32["sim"]
        torch.cuda.empty_cache()
        if not args.skip_err:
            fp32["err_vs_fp64"] = fp32_error_vs_fp64(fs, torch, device)

    ens = None
    if not args.skip_ensemble:
        ens = ensemble(fs, torch, args, hbm, peak_src)

    win = None
    if not args.skip_window:
        win = window(torch, args)

    e2e = end_to_end(fs, torch, device, args, dist, world)

    cpu = None
    if rank == 0 and not args.skip_cpu:
        cpu = cpu_baseline(args)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD_NAME, "grid": [4096, 256], "ppc": 16,
                       "n_particles": res64["n_mean"], "precision": "fp64",
                       "tiles": res64["tiles"], "tile": list(res64["tile"]),
                       "l2": "inputs larger than L2 (1.6 GB particle state per step)",
                       "parallelism": f"replicas x{world}"},
            "roofline": roofline,
            "fp32": fp32,
            "ensemble": ens,
            "window": win,
            "e2e": e2e,
            "cpu_baseline": cpu,
            "gpu_launches": gpu_launches,
            "clocks": res64["clocks"],
        }
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()


def ensemble(fs, torch, args, hbm, peak_src):
    """The batched ensemble: 64 uneven 1D FP32 runs stepped together (one
    push launch over every run's CTA group per step, graph-captured), timed
    with CUDA events, next to the same runs stepped one after another."""
    from paper_2507_14282_gb300 import tune
    from tests.workloads import config4_runs
    tuner = tune.Autotuner(widths=fs.FsBatch.COMPILED_WIDTHS)
    t0 = time.perf_counter()
    runs = [tuner.tile(r) for r in config4_runs(64)]
    tune_s = time.perf_counter() - t0
    sims = [fs.FauxShock(**r) for r in runs]
    st = sims[0].stream
    K = args.ens_steps
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    for s in sims:
        s.step(args.warmup)
    torch.cuda.synchronize()
    e0.record(st)
    for s in sims:
        s.step(K)
    e1.record(st)
    torch.cuda.synchronize()
    seq_ms = e0.elapsed_time(e1) / K
    n0 = sum(s.num_particles() for s in sims)
    b = fs.FsBatch(sims)
    b.step(args.warmup)
    torch.cuda.synchronize()
    e0.record(st)
    b.step(K)
    e1.record(st)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / K
    n1 = sum(s.num_particles() for s in sims)
    status = [s.diag()["status"] for s in sims]
    b.close()
    n = 0.5 * (n0 + n1)
    pb = particle_bytes(4, 1)
    grid_b = sum(GRID_WORDS_PER_CELL * 4 * (r["nx"] + 1) for r in runs)
    step_bytes = n * pb + grid_b
    for s in sims:
        s.close()
    torch.cuda.empty_cache()
    return {"workload": ENSEMBLE_NAME, "value": n / (ms * 1e-3), "unit": UNIT,
            "ms_per_step": ms, "steps": K, "n_runs": len(runs), "n_particles": n,
            "sequential_value": n / (seq_ms * 1e-3), "sequential_ms_per_step": seq_ms,
            "speedup_vs_sequential": seq_ms / ms,
            "bytes_per_particle_step": step_bytes / n,
            "step_roofline": {"bound": "hbm", "achieved": step_bytes / (ms * 1e-3) / 1e9,
                              "peak": hbm, "unit": "GB/s",
                              "frac": step_bytes / (ms * 1e-3) / 1e9 / hbm,
                              "peak_source": peak_src},
            "tiles": {k: v for k, v in sorted(tuner.cache.items())},
            "tune_s": tune_s, "status_ok": all(x == 0 for x in status)}


FIELD_NAMES = ("B", "E", "Bbar", "n", "J", "u")


def fp32_error_vs_fp64(fs, torch, device):
    """Relative L2 error of every field and moment of the FP32 precision form
    against the same box (8192 x 512 cells, 64 ppc, seed 3) run by the plain
    FP64 method on the GPU, after 1 and after 100 steps from fresh handles.
    "rel_l2" divides by the FP64 field's norm; "rel_l2_fluct" by the norm of
    its departure from the initial uniform state (B0, motional E, n = 1,
    u = -M_A x), the sharper figure for the fields that stay near it."""
    import numpy as np
    whats = (fs.FS_B, fs.FS_E, fs.FS_BBAR, fs.FS_N, fs.FS_J, fs.FS_U)
    f32 = fs.FauxShock(device=device, precision=fs.FS_FP32, **FP32_WORKLOAD)
    f64 = fs.FauxShock(device=device, precision=fs.FS_FP64, **FP32_WORKLOAD)
    g0 = [f64.grid(w) for w in whats]
    out = {}
    for label, k in (("after_1_step", 1), ("after_100_steps", 99)):
        f32.step(k)
        f64.step(k)
        a = [f32.grid(w) for w in whats]
        b = [f64.grid(w) for w in whats]
        rel = {n: float(np.linalg.norm(x - y) / np.linalg.norm(y))
               for n, x, y in zip(FIELD_NAMES, a, b)}
        fl = {n: float(np.linalg.norm(x - y) / max(np.linalg.norm(y - z), 1e-300))
              for n, x, y, z in zip(FIELD_NAMES, a, b, g0)}
        d32, d64 = f32.diag(), f64.diag()
        out[label] = {"rel_l2": rel, "rel_l2_fluct": fl,
                      "reflected": [d32["reflected"], d64["reflected"]],
                      "injected": [d32["injected"], d64["injected"]]}
    f32.close()
    f64.close()
    del f32, f64
    torch.cuda.empty_cache()
    out["reference"] = ("the same box in FP64 on the GPU (bit-exact to the FP64 oracle "
                        "in the parity tests)")
    out["tolerance"] = {"after_1_step": 1e-5, "after_100_steps": 1e-3}
    return out


WINDOW_NAME = ("differentiable window, 1D faux-shock box: 2048 cells, 128 ppc (262k ions), "
               "M_A=20, theta_Bn=0, beta=1, CR source p_iso=100 n_cr=0.01, 200 steps "
               "checkpointed every 20, loss = upstream |dB_perp|^2 dx, gradient w.r.t. 16 "
               "mode amplitudes, u_cr and u2; seed 4")


def window(torch, args):
    """The differentiable window (FP32 and FP64): forward, and forward +
    backward (each segment recomputed from its checkpoint, then the adjoint
    sweep), timed on the host around the synchronising calls."""
    import numpy as np
    from paper_2507_14282_gb300 import window as W
    from tests import window_inputs as WI
    X, V = WI.plasma(2048, 128)
    amps, ph = WI.modes()
    th = WI.theta(amps)
    out = {"workload": WINDOW_NAME, "unit": UNIT}
    for name, prec in (("fp32", 1), ("fp64", 0)):
        w = W.FauxShockWindow(X, V, ph, steps=200, ckpt=20, nx=2048, ny=1, ppc=128,
                              precision=prec, cr_enable=1, fs_mode_thermal=1, p_iso=100.0,
                              n_cr_ratio=0.01, **WI.COMMON)
        w.loss_and_grad(th)  # warm-up
        K = 3
        t0 = time.perf_counter()
        for _ in range(K):
            w.forward(th)
        tf = (time.perf_counter() - t0) / K
        t0 = time.perf_counter()
        for _ in range(K):
            L, g = w.loss_and_grad(th)
        tfb = (time.perf_counter() - t0) / K
        c = w.counts()
        n = 2048 * 128 + c["injected"] / 2  # mean slots over the window
        out[name] = {"forward_value": n * 200 / tf, "forward_backward_value": n * 200 / tfb,
                     "forward_ms": tf * 1e3, "forward_backward_ms": tfb * 1e3,
                     "loss": L, "grad_norm_modes": float(np.linalg.norm(g[:16])),
                     "grad_u_cr": float(g[16]), "grad_u2": float(g[17]),
                     "device_bytes": w.bytes, "counts": c}
        w.close()
        torch.cuda.empty_cache()
    return out


def end_to_end(fs, torch, device, args, dist, world):
    """The same metric through the public API with host buffers: the initial
    particle state is uploaded from pinned host memory (fs_inject), the steps
    run, and B, n and the diagnostics are read back to the host; all inside
    the timed region. Bytes are reported per step."""
    import numpy as np
    p = dict(FP64_WORKLOAD)
    nx, ny, ppc = p["nx"], p["ny"], p["ppc"]
    rng = np.random.default_rng(p["seed"])
    n = nx * ny * ppc
    pin = lambda a: torch.from_numpy(a).pin_memory().numpy()
    ci = pin(np.repeat(np.tile(np.arange(nx, dtype=np.int32), ny), ppc))
    cj = pin(np.repeat(np.repeat(np.arange(ny, dtype=np.int32), nx), ppc))
    fx = pin(rng.uniform(0, 1, n))
    fy = pin(rng.uniform(0, 1, n))
    vth = (p["beta_i"] / 2) ** 0.5
    vx = pin(rng.normal(-p["mach_a"], vth, n))
    vy = pin(rng.normal(0, vth, n))
    vz = pin(rng.normal(0, vth, n))
    steps = args.e2e_steps
    sim = fs.FauxShock(device=device, precision=fs.FS_FP64, init_plasma=0, **p)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    sim.inject(ci, cj, fx, fy, vx, vy, vz)
    sim.step(steps)
    B = sim.grid(fs.FS_B)
    nn = sim.grid(fs.FS_N)
    d = sim.diag()
    t1 = time.perf_counter()
    dt = t1 - t0
    if dist:
        tt = torch.tensor([dt], device=device)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        dt = float(tt.item())
    h2d = sum(a.nbytes for a in (ci, cj, fx, fy, vx, vy, vz))
    d2h = B.nbytes + nn.nbytes + 8 * 20
    val = 0.5 * (n + d["n_particles"]) * steps * world / dt
    sim.close()
    torch.cuda.empty_cache()
    return {"value": val, "unit": UNIT, "steps": steps,
            "h2d_bytes_per_step": h2d / steps, "d2h_bytes_per_step": d2h / steps,
            "wall_s": dt}


def cpu_baseline(args):
    """The FP64 CPU oracle, as it stands, on one host core, over a bounded
    sample of the workload: a 1/16 x-slice (256 x 256 cells, same ppc and
    physics) for a fixed number of steps."""
    from oracle import oracle as O
    p = dict(FP64_WORKLOAD)
    p["nx"] = 256
    sim = O.Oracle(**p)
    n0 = sim.num_particles
    steps = args.cpu_steps
    t0 = time.perf_counter()
    sim.step(steps)
    dt = time.perf_counter() - t0
    n1 = sim.num_particles
    sim.close()
    return {"value": 0.5 * (n0 + n1) * steps / dt, "unit": UNIT, "cores": 1,
            "kind": "oracle",
            "sample": f"256x256-cell x-slice of the FP64 workload (16 ppc, "
                      f"{n0} particles), {steps} steps, {dt:.1f} s, 1 core of "
                      f"{os.cpu_count()}"}


def reference(args):
    """The reference arm: the FP64 CPU oracle timed on the host on the same
    workload and metric, each step a bounded sample (a 1/16 x-slice)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import oracle as O
    p = dict(FP64_WORKLOAD)
    p["nx"] = 256
    sim = O.Oracle(**p)
    sim.step(args.warmup)
    n0 = sim.num_particles
    t0 = time.perf_counter()
    sim.step(args.steps)
    dt = time.perf_counter() - t0
    n1 = sim.num_particles
    sim.close()
    v = 0.5 * (n0 + n1) * args.steps / dt
    sample = (f"256x256-cell x-slice of the FP64 workload ({n0} particles) per step, "
              f"1 core of {os.cpu_count()}")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD_NAME, "sample": "1/16 x-slice (256x256 cells)"},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def ncu_case(args):
    """A small run of the benchmark's kernels for ncu captures, no timing:
    fp64 / fp32: the workload (on a smaller grid with --nx/--ny), init then
    --steps steps; ensemble: the 64-run batched ensemble (tiles from the
    autotuner), 3 batched steps then --steps more; window: one forward and
    one forward + backward of the differentiable window in FP32 (--steps
    window steps, checkpoints every 20)."""
    import torch
    from paper_2507_14282_gb300 import fs
    if args.ncu_case == "ensemble":
        from paper_2507_14282_gb300 import tune
        from tests.workloads import config4_runs
        runs = [tune.Autotuner(widths=fs.FsBatch.COMPILED_WIDTHS).tile(r) for r in config4_runs(64)]
        sims = [fs.FauxShock(**r) for r in runs]
        b = fs.FsBatch(sims)
        b.step(3)
        b.step(args.steps)
        torch.cuda.synchronize()
        ok = all(s.diag()["status"] == 0 for s in sims)
        b.close()
        print(json.dumps({"ncu_case": "ensemble", "runs": len(sims), "steps": 3 + args.steps,
                          "status_ok": ok}))
        return
    if args.ncu_case == "window":
        from paper_2507_14282_gb300 import window as Wn
        from tests import window_inputs as WI
        X, V = WI.plasma(2048, 128)
        amps, ph = WI.modes()
        w = Wn.FauxShockWindow(X, V, ph, steps=args.steps, ckpt=20, nx=2048, ny=1, ppc=128,
                               precision=1, cr_enable=1, fs_mode_thermal=1, p_iso=100.0,
                               n_cr_ratio=0.01, **WI.COMMON)
        th = WI.theta(amps)
        w.forward(th)
        L, g = w.loss_and_grad(th)
        w.close()
        print(json.dumps({"ncu_case": "window", "steps": args.steps, "loss": L}))
        return
    base = FP64_WORKLOAD if args.ncu_case == "fp64" else FP32_WORKLOAD
    p = dict(base)
    if args.nx:
        p["nx"] = args.nx
    if args.ny:
        p["ny"] = args.ny
    prec = fs.FS_FP64 if args.ncu_case == "fp64" else fs.FS_FP32
    sim = fs.FauxShock(precision=prec, capacity_factor=1.5, mover_fraction=0.1, **p)
    sim.step(args.steps)
    torch.cuda.synchronize()
    d = sim.diag()
    print(json.dumps({"ncu_case": args.ncu_case, "nx": p["nx"], "ny": p["ny"],
                      "steps": args.steps, "n_particles": d["n_particles"],
                      "status": d["status"]}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--ncu-case", choices=["fp64", "fp32", "ensemble", "window"], default=None,
                    help="run a small case of the benchmark kernels for ncu")
    ap.add_argument("--nx", type=int, default=0)
    ap.add_argument("--ny", type=int, default=0)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--steps32", type=int, default=50)
    ap.add_argument("--e2e-steps", type=int, default=50)
    ap.add_argument("--cpu-steps", type=int, default=300)
    ap.add_argument("--skip-fp32", action="store_true")
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--ens-steps", type=int, default=50)
    ap.add_argument("--skip-ensemble", action="store_true")
    ap.add_argument("--skip-window", action="store_true")
    ap.add_argument("--skip-err", action="store_true",
                    help="skip the FP32-vs-FP64 field error of the precision form")
    ap.add_argument("--prof-steps", type=int, default=20,
                    help="steps of the profiled pass that gives the phase timings")
    args = ap.parse_args()
    if args.ncu_case:
        ncu_case(args)
        return
    if args.warmup < 3:
        ap.error("--warmup must be at least 3")
    if args.impl == "reference":
        reference(args)
    else:
        ours(args)


if __name__ == "__main__":
    main()
