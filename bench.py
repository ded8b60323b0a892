"""Benchmark of the DiffWind hot path on GB300.

Headline workload (one "step"): the flag-like sheet at full size - 400,040
particles, 128^3 grid, Neo-Hookean E = 5e4, pinned edge, 32^3 x 16 Fourier
wind field, dt = 5e-5 - advanced by 1000 MLS-MPM substeps with a re-sort of
the particles by cell every 15 substeps, as one CUDA-graph replay. The metric
is MPM particle-substeps per second over all ranks (weak scaling: every rank
runs its own scene). Further measurements on the same run go into "metrics":
the MPM forward+adjoint rollout with checkpointing (100k-particle sheet on
64^3, 200 substeps, checkpoint every 20), the D3Q19 LBM step and its adjoint on
a 128^3 lattice with a leaf-cluster obstacle (MLUPS).

Timing: W untimed warm-up steps, then K steps each bracketed by CUDA events on
the launching stream; a 512 MB buffer is written between timed steps to flush
the 129 MB L2. `--impl reference` times the FP64 CPU oracle instead.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MPM particle-substeps/s fwd+adj, LBM MLUPS; surrogate vs plain LBM at stated error"
UNIT = "particle-substeps/s"
WORKLOAD = "sheet400k_128^3_1000substeps_fwd"
SORT_EVERY = 15


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--substeps", type=int, default=1000)
    ap.add_argument("--sort-every", type=int, default=SORT_EVERY,
                    help="substeps between particle re-sorts in the headline rollout")
    ap.add_argument("--no-extras", action="store_true", help="skip the secondary measurements")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--only", default=None, choices=["mpm", "lbm", "adjoint", "surrogate",
                                                    "surrogate_train", "batch",
                                                    "batch_adjoint", "inversion", "gsplat"],
                    help="run one part alone (for profiling): the sheet rollout, the 128^3 LBM "
                         "or the checkpointed MPM adjoint")
    ap.add_argument("--batch-scenes", type=int, default=64,
                    help="scenes of the batched workload (--only batch; 64 in the full run)")
    ap.add_argument("--p2g-mode", type=int, default=0,
                    help="P2G strategy: 0 auto, 1 global atomics, 2 warp-aggregated, 3 shared tile")
    return ap.parse_args()


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def reduce_max(x, device=None):
    """Max of a per-rank float over all ranks (the job's time is its slowest
    rank's); the value itself with one rank. device: where the reduction
    tensor lives (the rank's GPU under NCCL, the CPU under gloo)."""
    world, _, _ = dist_env()
    if world == 1:
        return float(x)
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(x)], dtype=torch.float64, device=device or "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(units_per_rank, world, ms_step):
    """Whole-job throughput: the units all ranks processed (replicas of the
    same workload, weak scaling) over the slowest rank's time."""
    return units_per_rank * world / (ms_step * 1e-3)


def replica_seeds(rank):
    """Seeds of rank r's replica: its own sheet jitter and wind field, the
    same workload shape on every rank."""
    return {"seed": rank, "wind_seed": rank}


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


# --------------------------------------------------------------- clocks ---

class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons while running."""
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200", "-f", self.path],
                stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            for ln in open(self.path):
                parts = [p.strip() for p in ln.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        except Exception:
            pass
        finally:
            try:
                os.unlink(self.path)
            except Exception:
                pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}

        def num(s):
            try:
                return float(s)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        smax = [num(r[2]) for r in rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        loaded = [v for v in sm if smax and v >= 0.5 * max(smax)] or sm
        return {"sm_mhz": statistics.median(loaded) if loaded else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": reasons, "samples": len(rows)}


# ------------------------------------------------------------- our arm ----

def run_ours(args):
    import torch

    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())

    from paper_2603_09668_gb300 import build as _build

    _build.build_library()
    from paper_2603_09668_gb300 import binding as B
    from paper_2603_09668_gb300 import inputs
    from paper_2603_09668_gb300.rollout import Rollout

    sc = inputs.sheet_scene(n_substeps=args.substeps, **replica_seeds(rank))
    n = sc.n
    mpm = B.MPM.from_params(sc.params(), max_particles=n, p2g_mode=args.p2g_mode)
    wind = B.WindField(torch.from_numpy(sc.wind).to(dev), sc.t_total)
    st0 = B.MpmState(*(torch.from_numpy(a).to(dev) for a in inputs.rest_state(sc.x)))
    pin0 = torch.from_numpy(sc.pinned).to(dev)
    ro = Rollout(mpm, n, wind, args.substeps, sort_every=args.sort_every, with_pins=True)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def step():
        ro.load(st0, pin0)
        ro.run()

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    mpm.device_status()

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    # ---- timed region: device time per step, L2 flushed between steps
    times = []
    barrier()
    wall0 = time.perf_counter()
    with ClockSampler(torch.cuda.current_device()) as clk:
        for _ in range(args.steps):
            flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step()
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
    barrier()
    wall = time.perf_counter() - wall0
    clocks = clk.summary()
    mpm.device_status()
    ms_step = reduce_max(sum(times) / len(times), dev)
    units = n * args.substeps * world
    value = job_value(n * args.substeps, world, ms_step)

    # ---- end to end through the public API: pinned host in, result out
    host_in = [a.cpu().pin_memory() for a in st0]
    host_pin = pin0.cpu().pin_memory()
    host_out = [torch.empty_like(a, device="cpu").pin_memory() for a in st0]
    host_ids = torch.empty(n, dtype=torch.int32).pin_memory()
    e2e_times = []
    dev_in = B.MpmState(*(torch.empty_like(a) for a in st0))
    dev_pin = torch.empty_like(pin0)
    for it in range(args.warmup + args.steps):
        flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for d, h in zip(dev_in, host_in):
            d.copy_(h, non_blocking=True)
        dev_pin.copy_(host_pin, non_blocking=True)
        ro.load(dev_in, dev_pin)
        res, ids = ro.run()
        for h, d in zip(host_out, res):
            h.copy_(d, non_blocking=True)
        host_ids.copy_(ids, non_blocking=True)
        e1.record(stream)
        e1.synchronize()
        if it >= args.warmup:
            e2e_times.append(e0.elapsed_time(e1))
    e2e_ms = reduce_max(sum(e2e_times) / len(e2e_times), dev)
    h2d = sum(a.numel() * a.element_size() for a in host_in) + host_pin.numel()
    d2h = sum(a.numel() * a.element_size() for a in host_out) + host_ids.numel() * 4

    # ---- roofline of the dominant kernel: per-kernel CUDA events over one
    # eager pass of the same rollout (same kernels, same inputs)
    ro_eager = Rollout(mpm, n, wind, args.substeps, sort_every=args.sort_every, with_pins=True,
                       use_graph=False)
    mpm.profile_enable(4 * args.substeps + 64)
    flush.fill_(1.0)
    ro_eager.load(st0, pin0)
    ro_eager.run()
    prof = mpm.profile_read()
    mpm.profile_enable(0)
    active_nodes = estimate_active_nodes(ro_eager, sc)
    fp32_peak = B.fp32_peak(paired=True) / 1e12  # FFMA2 throughput of this GPU, now
    roof = roofline(prof, n, active_nodes, fp32_peak)

    result = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "particles_per_gpu": n, "grid": sc.n_grid,
                   "substeps_per_step": args.substeps, "sort_every": args.sort_every,
                   "material": "neo-hookean E=5e4 nu=0.3", "wind": "32^3 x 16 Fourier",
                   "l2": "flushed between timed steps (512 MB write)", "p2g_mode": args.p2g_mode,
                   "parallelism": f"replicas x{world}"},
        "e2e": {"value": units / (e2e_ms * 1e-3), "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": ro.kernel_launches * args.steps,
        "clocks": clocks,
        "roofline": roof,
        "kernel_ms_per_launch": {k: (v[0] / v[1] if v[1] else None) for k, v in prof.items()},
        "wall_s_timed": wall,
    }
    if not args.no_extras:
        result["metrics"] = extras(dev, fp32_peak)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        result["cpu_baseline"] = cpu_baseline()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    if rank == 0:
        print(json.dumps(result), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def estimate_active_nodes(ro, sc):
    """Grid nodes inside the stencils of the final particle positions (for the
    per-node part of the algorithmic bytes)."""
    x = ro.result()[0].x.detach().cpu().numpy().astype(np.float64)
    N = sc.n_grid
    base = np.unique(np.floor(x * N - 0.5).astype(np.int64).T, axis=0)
    offs = np.stack(np.meshgrid(*[np.arange(3)] * 3, indexing="ij"), -1).reshape(-1, 3)
    nodes = (base[:, None, :] + offs[None, :, :]).reshape(-1, 3)
    lin = (nodes[:, 2] * N + nodes[:, 1]) * N + nodes[:, 0]
    return int(np.unique(lin).size)


# FP32 operations per particle-substep of the MLS-MPM substep, counted from
# its formulas (a multiply-add counts 2): stencil weights and their products
# for the old and the new position (2 x 87), G2P velocity (162) and affine
# matrix (657), position and deformation-gradient update (72), Neo-Hookean
# stress (62), affine momentum matrix (81), P2G mass and momentum of the 27
# nodes (783).
ALGO_FLOP_PER_PS = 1991

# DRAM bytes (read + write) of one launch of the fused kernel on the
# 400,040-particle sheet, from one ncu capture (dram__bytes_read.sum +
# dram__bytes_write.sum of the 5th launch of `bench.py --substeps 40 --steps 1
# --warmup 1 --no-extras --no-cpu-baseline`); valid only for the kernel
# sources it was taken on (hash of the files below), else reported as null.
G2P2G_TRAFFIC = {"sha16": "fcdfa04c31865798", "bytes": 20.10e6, "particles": 400040}
G2P2G_SOURCES = ("mpm_rollout.cu", "mpm_pair_warp.cuh", "mpm_pair.cuh", "mpm_p2g.cuh",
                 "mpm_math.cuh")


def g2p2g_source_sha():
    """Hash of the fused kernel's sources without their line comments and
    blank lines (an edited comment does not change the kernel the traffic
    was captured on)."""
    import hashlib
    import re

    h = hashlib.sha256()
    for f in G2P2G_SOURCES:
        with open(os.path.join(ROOT, "paper_2603_09668_gb300", "csrc", f), encoding="utf-8") as fh:
            code = re.sub(r"//[^\n]*", "", fh.read())
        h.update("\n".join(ln.rstrip() for ln in code.splitlines() if ln.strip()).encode())
    return h.hexdigest()[:16]


def hbm_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        return json.load(open(path))["hbm_gbs"], "MEASURED_PEAKS.json hbm_gbs (measured)"
    return 6800.0, "fallback 6.8 TB/s"


def roofline(prof, n, active_nodes, fp32_peak_tflops):
    """Roofline of the dominant kernel of the step, the fused G2P/P2G kernel
    (k_g2p2g_pair), from its average launch time (CUDA events over an eager
    pass of the same rollout). It is bound by instruction issue and latency:
    neither its DRAM traffic nor its FP32 pipe is saturated. `bound` names the
    nearer roof, the FP32 arithmetic: achieved = the method's FLOPs per
    launch (ALGO_FLOP_PER_PS x particles) over the launch time, peak = the
    FFMA2 throughput measured in this run. The HBM view is given beside it on
    two byte bases: the fused kernel's own (x and F read and written, 96 B per
    particle, plus 32 B per active node) and the unfused substep interface
    (x, v, C, F in and out, 192 B per particle, plus 56 B per active node)."""
    peak_gbs, peak_src = hbm_peak()
    ms, cnt = prof.get("g2p2g", (0.0, 0))
    if not cnt:
        return None
    avg_s = ms / cnt * 1e-3
    flops = ALGO_FLOP_PER_PS * n
    achieved = flops / avg_s / 1e12
    b_fused = 96 * n + 32 * active_nodes
    b_iface = 192 * n + 56 * active_nodes
    traffic = None
    if G2P2G_TRAFFIC["bytes"] and n == G2P2G_TRAFFIC["particles"] \
            and g2p2g_source_sha() == G2P2G_TRAFFIC["sha16"]:
        traffic = G2P2G_TRAFFIC["bytes"]
    return {"kernel": "g2p2g", "bound": "alu", "achieved": achieved, "peak": fp32_peak_tflops,
            "unit": "TFLOP/s", "frac": achieved / fp32_peak_tflops, "traffic": traffic,
            "algorithmic_flop_per_launch": flops, "avg_launch_us": avg_s * 1e6,
            "peak_source": "FFMA2 throughput probe (dw_fp32_probe), measured in this run",
            "hbm": {"peak_gbs": peak_gbs, "peak_source": peak_src,
                    "bytes_fused_basis": b_fused, "gbs_fused_basis": b_fused / avg_s / 1e9,
                    "frac_fused_basis": b_fused / avg_s / 1e9 / peak_gbs,
                    "bytes_interface_basis": b_iface,
                    "gbs_interface_basis": b_iface / avg_s / 1e9,
                    "frac_interface_basis": b_iface / avg_s / 1e9 / peak_gbs},
            "traffic_source": ("ncu dram bytes of one launch on the kernel sources of this run"
                               if traffic else "no capture of the current kernel sources")}


def roof_entry(rate, per_unit, peak, unit, bound, basis):
    """One workload's roofline line: achieved = rate x per_unit (in `unit`),
    frac = achieved / peak."""
    achieved = rate * per_unit
    return {"bound": bound, "achieved": achieved, "peak": peak, "unit": unit,
            "frac": achieved / peak, "basis": basis}


def _timed(fn, reps=3):
    import torch

    stream = torch.cuda.current_stream()
    fn()
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    return min(ts)


def bench_lbm(dev, steps=200, adj_steps=20):
    """D3Q19 step and adjoint on 128^3 with the leaf-cluster obstacle (200k
    particles in 50 ellipsoids, voxelized by Eq. point2voxel), tau = 0.55,
    inlet 0.05, and the HOME-LBM step on the same lattice. Algorithmic bytes:
    152 B per cell-step forward (BGK, 19 populations in and out), 80 B
    (HOME, 10 moments in and out)."""
    import torch

    from paper_2603_09668_gb300 import binding as B
    from paper_2603_09668_gb300 import inputs

    out = {}
    shape = (128, 128, 128)
    pts = torch.from_numpy(inputs.ellipsoid_cluster()).to(dev)
    solid = torch.empty((128, 128, 128), dtype=torch.uint8, device=dev)
    B.voxelize_particles(pts, shape, 1.0 / 128, solid)
    lbm = B.LBM(shape, 0.55, u_inlet=(0.05, 0.0, 0.0), bc_x=1, max_tape=max(adj_steps, 1))
    f = lbm.lattice(dev)
    ms = _timed(lambda: lbm.step(f, solid, steps))
    cells = 128 ** 3
    out["lbm_128_fwd_mlups"] = cells * steps / (ms * 1e-3) / 1e6
    out["lbm_128_fwd_gbs"] = 152 * cells * steps / (ms * 1e-3) / 1e9
    if adj_steps:
        g = torch.randn_like(f)
        ms = _timed(lambda: lbm.step_adjoint(f, g, solid, adj_steps))
        out["lbm_128_adj_mlups"] = cells * adj_steps / (ms * 1e-3) / 1e6
    # HOME-LBM on the same lattice: ten moments per cell, 40 B read + 40 B written
    m = lbm.moments(dev)
    lbm.home_init(m, 1.0, (0.05, 0.0, 0.0))
    home_steps = steps + (steps & 1)  # even: no copy back
    ms = _timed(lambda: lbm.home_step(m, solid, home_steps))
    out["lbm_128_home_mlups"] = cells * home_steps / (ms * 1e-3) / 1e6
    out["lbm_128_home_gbs"] = 80 * cells * home_steps / (ms * 1e-3) / 1e9
    lbm.close()
    return out


def bench_adjoint(dev):
    """MPM forward + adjoint with checkpointing: the 100k-particle sheet on 64^3,
    200 substeps, checkpoint every 20, loss on positions at the checkpoints,
    gradients with respect to the 32^3 x 16 wind grid and E."""
    import torch

    from paper_2603_09668_gb300 import autograd as AG
    from paper_2603_09668_gb300 import binding as B
    from paper_2603_09668_gb300 import inputs

    sc = inputs.sheet_scene(nu=274, nv=183, n_grid=64, n_substeps=200, dt=5e-5, seed=0,
                            wind_seed=0)
    mpm = B.MPM.from_params(sc.params(), max_particles=sc.n)
    st = B.MpmState(*(torch.from_numpy(a).to(dev) for a in inputs.rest_state(sc.x)))
    pin = torch.from_numpy(sc.pinned).to(dev)
    wv = torch.from_numpy(sc.wind).to(dev).requires_grad_(True)
    E = torch.tensor(sc.E, device=dev, requires_grad=True)
    target = torch.zeros((10, 3, sc.n), device=dev)

    def fwd_adj():
        X = AG.mpm_frames(mpm, st, wv, sc.t_total, E, 200, 20, pinned=pin)
        loss = ((X - target) ** 2).sum() / sc.n
        loss.backward()

    ms = _timed(fwd_adj, reps=2)
    mpm.close()
    return {"mpm_adj_sheet100k_64_ps_per_s": sc.n * 200 / (ms * 1e-3),
            "mpm_adj_note": "200 substeps forward + checkpointed adjoint (recompute + reverse)"}


SURR_CHECK_EVERY = 3  # the check interval that keeps the run within 2% (measured)


def bench_surrogate(dev, N=128, t_eval=1500, blocks=25, check_every=SURR_CHECK_EVERY):
    """The learned LBM surrogate on a held-out leaf-cluster scene (128^3, tau
    0.55, inlet 0.05 in a random direction), over the window t = 1500 -> 2000
    (25 blocks of 20 lattice steps) against the plain LBM trajectory:
      * one block: relative L2 velocity error of the network and of
        persistence (du = 0), the block times (surrogate chained block, plain
        block) and their ratio;
      * the run with the plain-LBM check every `check_every` blocks (the run
        goes on from the plain lattice after each check; above 2% the plain
        LBM takes over): final error against the plain trajectory, check
        errors, and the speed-up of the whole run against 25 plain blocks;
        the same run with persistence in place of the network (what the
        network gains at the same cost of checks);
      * the network chained over all 25 blocks without checks (its drift)."""
    import math

    import torch

    from paper_2603_09668_gb300 import binding as B
    from paper_2603_09668_gb300 import surrogate as S

    if not os.path.exists(S.weights_path(N)):
        return {"surrogate": "no trained weights"}
    rng = np.random.default_rng(987654)
    d = S.inlet_direction(rng)
    solid = S.leaf_mask(N, 424242, dev)
    m = S.SurrogateLBM(N, u_inlet=tuple(S.U_REF * d), check_every=check_every)
    f0 = m.lbm.lattice(dev)
    m.lbm.step(f0, solid, t_eval)
    ref = f0.clone()
    m.plain_block(ref, solid)
    err_persist = m.velocity_error(f0, ref, solid)
    m.surr.features(f0, solid, S.IN_SCALE)
    m.chained_block(solid)
    err_net = m.fine_error(ref, solid)
    # per-block times over runs of consecutive blocks (the steady state of a
    # run; one event pair per run, so no per-block host gap is counted)
    f = f0.clone()
    reps = 10
    ms_plain = _timed(lambda: [m.plain_block(f, solid) for _ in range(reps)], reps=2) / reps
    # the default mode: eager launches, every kernel a programmatic dependent
    # of the previous one, also across blocks
    m.surr.features(f0, solid, S.IN_SCALE)
    m.use_graph = False
    ms_surr = _timed(lambda: [m.chained_block(solid) for _ in range(reps)], reps=2) / reps
    # the same blocks replayed from a CUDA graph (first block eager, then captured)
    m.use_graph = True
    m.chained_block(solid)
    m.chained_block(solid)
    ms_surr_graph = _timed(lambda: [m.chained_block(solid) for _ in range(reps)], reps=2) / reps
    m.use_graph = False
    # the plain trajectory of the window, and the runs with checks
    f_plain = f0.clone()
    ms_plain_run = _timed(lambda: (f_plain.copy_(f0), m.lbm.step(f_plain, solid, 20 * blocks)), reps=1)
    out = {}
    for tag, pers in (("", False), ("_persistence", True)):
        m.persistence = pers
        f_sur = f0.clone()
        used = []

        def run():
            f_sur.copy_(f0)
            m.reset()
            used.append(m.advance(f_sur, solid, blocks))

        ms_run = _timed(run, reps=1)
        out[f"surr_run{tag}_final_err_vs_plain_trajectory"] = m.velocity_error(f_sur, f_plain, solid)
        out[f"surr_run{tag}_check_errors"] = m.errors
        out[f"surr_run{tag}_fallback"] = m.fallback
        out[f"surr_run{tag}_used"] = used[-1]
        out[f"surr_run{tag}_ms"] = ms_run
        out[f"surr_run{tag}_speedup"] = ms_plain_run / ms_run
    m.persistence = False
    # the network chained through the whole window without checks
    f_plain.copy_(f0)
    m.surr.features(f0, solid, S.IN_SCALE)
    drift = []
    for k in range(blocks):
        m.chained_block(solid)
        m.plain_block(f_plain, solid)
        if (k + 1) % 5 == 0:
            drift.append(m.fine_error(f_plain, solid))
    m.close()
    return {"surr_block_err": err_net, "persistence_err": err_persist,
            "surr_block_ms": ms_surr, "surr_block_graph_ms": ms_surr_graph,
            "plain_block_ms": ms_plain, "surr_speedup": ms_plain / ms_surr,
            "surr_run_blocks": blocks, "surr_run_check_every": check_every,
            "plain_run_ms": ms_plain_run, **out,
            "surr_chain_no_check_err_every5": drift,
            "surr_note": ("window t = 1500 -> 2000 of a held-out scene; run = network blocks with "
                          f"the plain-LBM check every {check_every} blocks (continuing from the "
                          "plain lattice); _persistence = the same run with du = 0")}


def bench_batch(dev, n_scenes=64, n_sub=500, sort_every=25, trial=10):
    """64 uneven scenes (particle counts log-uniform 20k-400k, 64^3 / 128^3
    grids, sheets and blocks, each with its own 16^3 x 8 wind) advanced by the
    batched rollout: one launch per substep, replayed from a CUDA graph, launch
    shape picked by the autotuner. Reported: whole-batch particle-substeps/s
    over n_sub substeps with re-sorting every sort_every, and the tuner's
    table (ms per substep per candidate)."""
    import torch

    from paper_2603_09668_gb300 import binding as B
    from paper_2603_09668_gb300 import inputs

    scenes = inputs.batch_scenes(n_scenes=n_scenes, n_substeps=n_sub)
    winds = [B.WindField(torch.from_numpy(sc.wind.astype(np.float32)).to(dev), sc.t_total)
             for sc in scenes]
    batch = B.MPMBatch([(sc.params(), sc.n, w) for sc, w in zip(scenes, winds)])
    st = [np.concatenate([inputs.rest_state(sc.x)[i] for sc in scenes], axis=1) for i in range(4)]
    pin = np.concatenate([sc.pinned if sc.pinned is not None else np.zeros(sc.n, np.uint8)
                          for sc in scenes])
    s0 = B.MpmState(*(torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in st))
    p0 = torch.from_numpy(pin).to(dev)
    best, trials = batch.tune(s0, p0, n_trial_substeps=trial)
    s = s0.clone()
    p = p0.clone()
    ids = torch.arange(batch.n, dtype=torch.int32, device=dev)

    def run():
        batch.rollout(s, p, ids, 0.0, n_sub, sort_every)

    ms = _timed(run, reps=2)
    batch.device_status()
    cfg = batch.config()
    batch.close()
    n = int(batch.n)
    return {"batch_scenes": n_scenes, "batch_particles": n, "batch_substeps": n_sub,
            "batch_ps_per_s": n * n_sub / (ms * 1e-3), "batch_ms_per_substep": ms / n_sub,
            "batch_config": cfg, "batch_tuner": [[t[0]["mode"], t[0]["threads"],
                                                  t[0]["ctas_per_sm"], round(t[1], 4)]
                                                 for t in trials]}


def bench_batch_adjoint(dev, n_scenes=64, n_sub=500, ckpt=25, trial=10):
    """Batched forward + adjoint of the 64-scene workload: the forward rollout
    of n_sub substeps in segments of ckpt substeps, each segment's start state
    stored as a checkpoint; then, from dL/d(final state) (a fixed seed
    gradient), the reverse pass of every segment in reverse order by
    mpm_batch_segment_adjoint (recomputing the segment's states into a tape),
    accumulating each scene's wind and E gradients. Reported: whole-batch
    particle-substeps/s of forward + adjoint together, and of the reverse
    pass alone."""
    import torch

    from paper_2603_09668_gb300 import binding as B
    from paper_2603_09668_gb300 import inputs

    scenes = inputs.batch_scenes(n_scenes=n_scenes, n_substeps=n_sub)
    winds = [B.WindField(torch.from_numpy(sc.wind.astype(np.float32)).to(dev), sc.t_total)
             for sc in scenes]
    batch = B.MPMBatch([(sc.params(), sc.n, w) for sc, w in zip(scenes, winds)])
    st = [np.concatenate([inputs.rest_state(sc.x)[i] for sc in scenes], axis=1) for i in range(4)]
    pin = np.concatenate([sc.pinned if sc.pinned is not None else np.zeros(sc.n, np.uint8)
                          for sc in scenes])
    s0 = B.MpmState(*(torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in st))
    p = torch.from_numpy(pin).to(dev)
    batch.tune(s0, p, n_trial_substeps=trial)
    n = int(batch.n)
    dt = scenes[0].dt
    assert all(sc.dt == dt for sc in scenes)
    n_seg = n_sub // ckpt
    s = s0.clone()
    ck = [B.MpmState.empty_like(s0) for _ in range(n_seg)]
    tape = torch.empty((ckpt - 1) * 24 * n, dtype=torch.float32, device=dev)
    g = B.MpmState.empty_like(s0)
    g0 = B.MpmState.zeros_like(s0)
    g0.x.fill_(1.0 / n)  # L = mean of the final positions' coordinates
    nw, _ = batch.wind_layout()
    g_wind = torch.zeros(nw, dtype=torch.float32, device=dev)
    g_E = torch.zeros(n_scenes, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    marks = {}

    def run():
        for a, b in zip(s, s0):
            a.copy_(b)
        for i in range(n_seg):
            for a, b in zip(ck[i], s):
                a.copy_(b)
            batch.rollout(s, p, None, i * ckpt * dt, ckpt, 0)
        marks["mid"] = torch.cuda.Event(enable_timing=True)
        marks["mid"].record(stream)
        for a, b in zip(g, g0):
            a.copy_(b)
        for i in reversed(range(n_seg)):
            batch.segment_adjoint(ck[i], tape, g, p, i * ckpt * dt, ckpt, g_wind, g_E)
        marks["end"] = torch.cuda.Event(enable_timing=True)
        marks["end"].record(stream)

    ms = _timed(run, reps=1)
    adj_ms = marks["mid"].elapsed_time(marks["end"])
    batch.device_status()
    finite = bool(torch.isfinite(g_wind).all().item() and torch.isfinite(g_E).all().item())
    cfg = batch.config()
    batch.close()
    return {"batch_adj_scenes": n_scenes, "batch_adj_particles": n, "batch_adj_substeps": n_sub,
            "batch_adj_checkpoint_every": ckpt,
            "batch_fwd_adj_ps_per_s": n * n_sub / (ms * 1e-3),
            "batch_adj_only_ps_per_s": n * n_sub / (adj_ms * 1e-3),
            "batch_fwd_adj_ms": ms, "batch_adj_ms": adj_ms, "batch_adj_grads_finite": finite,
            "batch_adj_config": cfg}


def bench_inversion(dev, iters=40):
    """The physics-informed wind inversion (Sec. 3.3, 3.4) on the synthetic
    flag case (5,504 particles on 64^3, 12^3 wind grid, 32^3 guide lattice,
    3 intervals of 200 substeps at dt 2e-4, checkpoint every 25): one Adam
    iteration = 200 substeps forward + checkpointed adjoint + L_phys +
    VectorAdam. Scores against the ground-truth drag field (App. E.2) with and
    without L_phys."""
    import torch

    from paper_2603_09668_gb300 import inputs
    from paper_2603_09668_gb300 import inversion as I

    case = inputs.inversion_case()
    out = {}
    for lam, tag in ((0.1, ""), (0.0, "_no_phys")):
        syn = I.prepare_synthetic(case, dev)
        inv = I.WindInversion(syn.mpm, syn.guide, case["substeps"], case["every"], iters, 1.0, lam)
        stream = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        res = inv.reconstruct(syn.state0, syn.pinned, syn.x_obs, case["lbm_steps"])
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        cos, nmse = I.field_scores(res.values, syn.gt_forces)
        syn.close()
        out[f"inversion_cos_sim{tag}"] = cos
        out[f"inversion_nmse{tag}"] = nmse
        if not tag:
            n_it = case["n_intervals"] * iters
            out["inversion_iter_ms"] = ms / n_it
            out["inversion_ps_per_s"] = case["scene"].n * case["substeps"] * n_it / (ms * 1e-3)
            out["inversion_total_ms"] = ms
    # observed through two rendered 128 x 128 views instead of the particle positions
    for lam, tag in ((0.1, ""), (0.0, "_no_phys")):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res = I.run_synthetic(case, iters=iters, lr=1.0, lam_phys=lam, observe="render")
        torch.cuda.synchronize()
        out[f"inversion_render_cos_sim{tag}"] = res["cos_sim"]
        out[f"inversion_render_nmse{tag}"] = res["nmse"]
        if not tag:
            out["inversion_render_wall_s"] = time.perf_counter() - t0
    out["inversion_note"] = (f"{case['scene'].n} particles, 64^3 grid, 12^3 wind grid, "
                             f"{case['n_intervals']} intervals x {iters} iterations x "
                             f"{case['substeps']} substeps (forward + adjoint), guide inlet "
                             f"{case['inlet_error_deg']} deg off; lambda_phys 0.1; render: two 128 x 128 views, "
                             f"0.9 L1 + 0.1 D-SSIM, wall time includes the ground truth and "
                             f"its images")
    return out


def bench_gsplat(dev):
    """Particle-bound Gaussian splatting: the 100,284-particle sheet (64^3
    case) drawn at 512 x 512, forward (covariance update, projection, depth
    sort, tile compositing) and reverse mode (down to dL/dx and dL/dF)."""
    import torch

    from paper_2603_09668_gb300 import binding as B
    from paper_2603_09668_gb300 import inputs

    sc = inputs.sheet_scene(nu=274, nv=183, n_grid=64, n_substeps=1, seed=0)
    n = sc.n
    g = np.random.default_rng(7)
    F = np.zeros((9, n), np.float32)
    F[[0, 4, 8]] = 1.0
    F += g.uniform(-0.05, 0.05, (9, n)).astype(np.float32)
    s0 = np.zeros((6, n), np.float32)
    s0[:3] = 0.003 ** 2
    arrs = [torch.from_numpy(a).to(dev) for a in
            (sc.x, F, s0, g.uniform(0, 1, (3, n)).astype(np.float32),
             g.uniform(0.3, 0.9, n).astype(np.float32))]
    cam = B.camera(np.eye(3), (-0.5, -0.6, 1.2), 600.0, 600.0, 256.0, 256.0, 512, 512)
    r = B.GaussianRenderer(n, 512, 512)
    img = torch.empty((3, 512, 512), device=dev)
    g_img = torch.randn((3, 512, 512), device=dev)
    g_x, g_F = torch.zeros_like(arrs[0]), torch.zeros_like(arrs[1])
    fwd_ms = _timed(lambda: r.render(cam, *arrs, image=img))
    bwd_ms = _timed(lambda: r.backward(cam, *arrs, g_img, g_x, g_F))
    r.close()
    return {"gs_sheet100k_512_fwd_ms": fwd_ms, "gs_sheet100k_512_bwd_ms": bwd_ms,
            "gs_gaussians": n}


def bench_surrogate_train(dev, n=64, reps=10):
    """One training step of the surrogate network at 64^3 coarse voxels
    (forward keeping the activations, MSE loss, reverse pass, Adam), its
    reverse pass alone, and each layer shape's weight-gradient kernel on
    tcgen05 and on mma.sync (surr_weight_grad), with their FLOP rates
    (2 x 27 x cin x cout per voxel)."""
    import numpy as np
    import torch

    from paper_2603_09668_gb300 import binding as B

    s = B.Surrogate(n)
    rng = np.random.default_rng(0)
    s.set_params(torch.tensor(rng.standard_normal(s.nparams).astype(np.float32) * 0.05).to(dev))
    s.set_features(torch.tensor(rng.standard_normal((n ** 3, 16)).astype(np.float32)).to(dev))
    out = torch.empty((n ** 3, 16), device=dev)
    target = torch.tensor(rng.standard_normal((n ** 3, 16)).astype(np.float32) * 0.1).to(dev)
    loss = torch.zeros(1, device=dev)
    step = [0]

    def train_step():
        step[0] += 1
        s.zero_grads()
        s.forward(out, keep_activations=True)
        s.loss(target, loss)
        s.backward()
        s.adam(1e-4, step=step[0])

    res = {"surr_train_step_ms": _timed(train_step, reps), "surr_backward_ms": _timed(s.backward, reps)}
    for cin, cout in ((16, 32), (32, 32), (32, 16)):
        x = torch.randn((cin // 8, n ** 3, 8), device=dev).to(torch.bfloat16).contiguous()
        g = torch.randn((cout // 8, n ** 3, 8), device=dev).to(torch.bfloat16).contiguous()
        gw = torch.zeros(27 * cin * cout, device=dev)
        gb = torch.zeros(cout, device=dev)
        flop = 2 * 27 * cin * cout * n ** 3
        for impl, name in ((0, "tc"), (1, "mma")):
            ms = _timed(lambda: s.weight_grad(cin, cout, x, g, gw, gb, impl=impl), reps)
            res[f"surr_wgrad_{cin}_{cout}_{name}_us"] = ms * 1e3
            res[f"surr_wgrad_{cin}_{cout}_{name}_tflops"] = flop / ms / 1e9
    s.device_status()
    s.close()
    res["surr_train_note"] = ("64^3 coarse voxels; wgrad: one layer's weight and bias gradients, "
                              "tc = tcgen05 (the kernel the reverse pass runs), mma = mma.sync")
    return res


def extras(dev, fp32_peak):
    out = bench_lbm(dev)
    out.update(bench_adjoint(dev))
    out.update(bench_surrogate(dev))
    out.update(bench_surrogate_train(dev))
    out.update(bench_batch(dev))
    out.update(bench_batch_adjoint(dev))
    out.update(bench_inversion(dev))
    out.update(bench_gsplat(dev))
    out["roofline"] = workload_rooflines(out, fp32_peak)
    return out


def workload_rooflines(m, fp32_peak):
    """Roofline lines of the secondary workloads from their measured rates:
    bytes per unit are the algorithmic interface bytes (LBM: populations or
    moments in and out; MPM: particle state in and out), FLOPs per call of the
    surrogate are those of the network the method specifies."""
    gbs, _ = hbm_peak()
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) \
        if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    bf16 = peaks.get("bf16_tflops", 1900.0)
    r = {}
    if "lbm_128_fwd_mlups" in m:
        r["lbm_128_fwd"] = roof_entry(m["lbm_128_fwd_mlups"] * 1e6, 152 / 1e9, gbs, "GB/s", "hbm",
                                      "152 B per cell-step (19 populations in and out)")
    if "lbm_128_adj_mlups" in m:
        r["lbm_128_adj"] = roof_entry(m["lbm_128_adj_mlups"] * 1e6, 380 / 1e9, gbs, "GB/s", "hbm",
                                      "380 B per cell-step (state, adjoint in and out: 228; "
                                      "the forward recompute: 152)")
    if "lbm_128_home_mlups" in m:
        r["lbm_128_home"] = roof_entry(m["lbm_128_home_mlups"] * 1e6, 80 / 1e9, gbs, "GB/s", "hbm",
                                       "80 B per cell-step (10 moments in and out)")
    if "mpm_adj_sheet100k_64_ps_per_s" in m:
        r["mpm_fwd_adj_sheet100k_64"] = roof_entry(
            m["mpm_adj_sheet100k_64_ps_per_s"], 672 / 1e9, gbs, "GB/s", "hbm",
            "672 B per particle-substep (forward 192; reverse 480: recompute 192, stored "
            "state 96, adjoint state in and out 192)")
    if "batch_ps_per_s" in m:
        r["batch_fwd"] = roof_entry(m["batch_ps_per_s"], 192 / 1e9, gbs, "GB/s", "hbm",
                                    "192 B per particle-substep (x, v, C, F in and out)")
        r["batch_fwd_flops"] = roof_entry(m["batch_ps_per_s"], ALGO_FLOP_PER_PS / 1e12, fp32_peak,
                                          "TFLOP/s", "alu", f"{ALGO_FLOP_PER_PS} FLOP per "
                                          "particle-substep, FFMA2 peak measured in this run")
    if "batch_fwd_adj_ps_per_s" in m:
        r["batch_fwd_adj"] = roof_entry(m["batch_fwd_adj_ps_per_s"], 672 / 1e9, gbs, "GB/s", "hbm",
                                        "672 B per particle-substep (as the single-scene adjoint)")
    if "surr_block_ms" in m:
        r["surrogate_block"] = roof_entry(1.0 / (m["surr_block_ms"] * 1e-3), 32.6e9 / 1e12, bf16,
                                          "TFLOP/s", "tensor",
                                          "32.6 GFLOP per call (5 -> 32 -> 32 -> 32 -> 3 channels, "
                                          "kernel 3, 64^3; the kernels run 16-channel padded ends, "
                                          "43.5 GFLOP) over the whole block (network and "
                                          "chained update); BF16 burst peak of MEASURED_PEAKS.json")
    if "surr_wgrad_32_32_tc_us" in m:
        r["surrogate_wgrad_32_32"] = roof_entry(1.0 / (m["surr_wgrad_32_32_tc_us"] * 1e-6),
                                                2 * 27 * 32 * 32 * 64 ** 3 / 1e12, bf16, "TFLOP/s",
                                                "tensor",
                                                "one 32 -> 32 layer's weight gradient at 64^3 "
                                                "(14.5 GFLOP, tcgen05, bias and partial-sum "
                                                "reduction included); BF16 burst peak")
    return r


def _oracle_sheet_run(args):
    """Runs n_sub FP64 oracle substeps of the full sheet (replica `seed`) in
    this process and returns the seconds taken (one replica per host core)."""
    n_sub, seed = args
    import oracle
    from paper_2603_09668_gb300 import inputs

    sc = inputs.sheet_scene(seed=seed, wind_seed=seed)
    st = tuple(a.astype(np.float64) for a in inputs.rest_state(sc.x))
    t0 = time.perf_counter()
    for k in range(n_sub):
        st = oracle.mpm_substep(sc.params(), st, sc.wind_tuple(), k * sc.dt, sc.pinned)
    return time.perf_counter() - t0


def _oracle_lbm_run(args):
    """Runs `steps` FP64 oracle BGK steps of the 128^3 leaf-cluster lattice
    (tau 0.55, inlet 0.05 along x) in this process; returns the seconds."""
    steps, seed = args
    import oracle
    from paper_2603_09668_gb300 import inputs

    shape = (128, 128, 128)
    solid = oracle.voxelize(inputs.ellipsoid_cluster(seed=seed), shape, 1.0 / 128)
    _, w, _ = oracle.velocity_set()
    f = np.repeat(w[:, None], 128 ** 3, axis=1)
    t0 = time.perf_counter()
    oracle.lbm_step(shape, 0.55, f, steps, u_in=(0.05, 0.0, 0.0), bc_x=1, solid=solid)
    return time.perf_counter() - t0


def cpu_baseline(n_sub=75, n_sub_all=30, lbm_steps=4):
    """The FP64 oracle on this host: n_sub substeps of the full 400k sheet on
    one core, and independent replicas of n_sub_all substeps on every core at
    once (processes started with spawn), the whole job's rate reported; and
    lbm_steps BGK steps of the 128^3 leaf-cluster lattice the same two ways,
    in MLUPS."""
    import multiprocessing

    import oracle
    from paper_2603_09668_gb300 import inputs

    oracle.build()
    n = inputs.sheet_scene().n
    one = _oracle_sheet_run((n_sub, 0))
    cores = host_cores()
    ctx = multiprocessing.get_context("spawn")
    with ctx.Pool(cores) as pool:
        pool.map(_oracle_sheet_run, [(1, r) for r in range(cores)])  # load the library once
        t0 = time.perf_counter()
        pool.map(_oracle_sheet_run, [(n_sub_all, r) for r in range(cores)])
        wall = time.perf_counter() - t0
        # the LBM step: one core, then one replica per core
        lbm_one = _oracle_lbm_run((lbm_steps, 0))
        t0 = time.perf_counter()
        pool.map(_oracle_lbm_run, [(lbm_steps, r) for r in range(cores)])
        lbm_wall = time.perf_counter() - t0
    cells = 128 ** 3
    return {"value": cores * n * n_sub_all / wall, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": (f"{cores} independent replicas (one per core) of {n_sub_all} substeps of the "
                       f"full 400,040-particle sheet on 128^3 (FP64, serial C each)"),
            "seconds": wall,
            "one_core": {"value": n * n_sub / one, "cores": 1,
                         "sample": f"{n_sub} substeps of the full sheet on one core", "seconds": one},
            "lbm_128": {"unit": "MLUPS", "one_core": cells * lbm_steps / lbm_one / 1e6,
                        "all_cores": cores * cells * lbm_steps / lbm_wall / 1e6, "cores": cores,
                        "sample": (f"{lbm_steps} FP64 oracle BGK steps of the 128^3 leaf-cluster "
                                   f"lattice on one core, then one replica per core")}}


# ------------------------------------------------------- reference arm ----

def run_reference(args):
    """The FP64 oracle on the host's cores: every step, one independent
    replica of the full sheet per core (processes started with spawn) runs
    3 substeps; value = particle-substeps of all replicas per second."""
    world, rank, _ = dist_env()
    if rank != 0:
        return
    import multiprocessing

    import oracle
    from paper_2603_09668_gb300 import inputs

    oracle.build()
    n = inputs.sheet_scene().n
    n_sub = 3  # each step: 3 substeps of the full sheet per core (~1-2 s of FP64 CPU work)
    cores = host_cores()
    ctx = multiprocessing.get_context("spawn")
    with ctx.Pool(cores) as pool:
        def step():
            pool.map(_oracle_sheet_run, [(n_sub, r) for r in range(cores)])

        pool.map(_oracle_sheet_run, [(1, r) for r in range(cores)])  # load the library once
        for _ in range(args.warmup):
            step()
        ts = []
        for _ in range(args.steps):
            t0 = time.perf_counter()
            step()
            ts.append(time.perf_counter() - t0)
    s_step = sum(ts) / len(ts)
    value = cores * n * n_sub / s_step
    sample = (f"{cores} independent replicas (one per core) of {n_sub} substeps of the full "
              f"400,040-particle sheet on 128^3 per step (FP64, serial C each)")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": s_step * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD, "reference": "FP64 CPU oracle"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def run_only(args):
    import torch

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    from paper_2603_09668_gb300 import build as _build

    _build.build_library()
    if args.only == "lbm":
        res = bench_lbm(dev, steps=2 * max(args.steps, 1), adj_steps=2)
    elif args.only == "surrogate":
        res = bench_surrogate(dev)
    elif args.only == "surrogate_train":
        res = bench_surrogate_train(dev)
    elif args.only == "batch":
        res = bench_batch(dev, n_scenes=args.batch_scenes)
    elif args.only == "batch_adjoint":
        res = bench_batch_adjoint(dev, n_scenes=args.batch_scenes)
    elif args.only == "inversion":
        res = bench_inversion(dev)
    elif args.only == "gsplat":
        res = bench_gsplat(dev)
    else:
        res = bench_adjoint(dev)
    print(json.dumps({"only": args.only, **res}), flush=True)


if __name__ == "__main__":
    a = parse()
    if a.impl == "reference":
        run_reference(a)
    elif a.only in ("lbm", "adjoint", "surrogate", "surrogate_train", "batch", "batch_adjoint",
                    "inversion", "gsplat"):
        run_only(a)
    else:
        run_ours(a)
