"""Benchmark of the EAM timestep on GB300.

Workload: the 799,496-atom BCC system (74x74x73 cells, Johnson-form EAM,
2,000-knot cubic tables, r_cut 4.5 A, skin 0.3 A, sigma 0.02 A, 300 K),
mixed precision (FP32 pair arithmetic; FP64 positions, velocities,
integration and sums), dt = 2 fs, list rebuilt every 10 steps.

One benchmark "step" is one pass of the whole hot path: 10 velocity-Verlet
timesteps (a list rebuild: wrap, bin, sort, permute, list; ten density and
force/integration passes) plus one energy/virial evaluation.  The metric is
MD timesteps per second (higher is better).

  value   device-timed throughput with the state resident in HBM (CUDA events
          on the library's stream, K steps after W warm-up steps; the working
          set, ~0.35 GB, is larger than L2, so no flush is needed)
  e2e     the same metric through the C ABI with host buffers: per step
          md_set_state from pinned host memory (positions + velocities),
          md_step(10), md_energy (reads PE and KE back)

After the timed region (rank 0, one GPU) the line also carries short legs
measured in the same run: the plain FP64 GPU path on the same system
(`fp64`, and the mixed/FP64 ratio), the half-list form (`half_list`), the
512-replica batched launch (`batch`, atom-steps/s), the force-matching
gradient (`adjoint`: seconds per loss and gradient, and its agreement with
finite differences) and the oracle on all host cores
(`cpu_baseline_all_cores`); --no-extras leaves them out.

--impl reference times the CPU oracle (the plain serial FP64 C reference)
on a bounded sample of the same workload: one timestep per benchmark step.
With torchrun (N > 1) every rank advances its own replica of the system
(the single-system path does not shard across GPUs) and rank 0 reports the
sum over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

MD_STEPS_PER_BENCH_STEP = 10
DT_FS = 2.0
WORKLOAD = "bcc_799496_mixed"


def _dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            p = json.load(fh)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.rows = []
        self._proc = None
        self._thread = None

    def start(self):
        try:
            self._proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "10"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self._proc = None
            return
        self._thread = threading.Thread(target=self._read, daemon=True)
        self._thread.start()
        # the timed region starts once the sampler is live
        t0 = time.time()
        while not self.rows and time.time() - t0 < 3.0:
            time.sleep(0.01)

    def mark(self):
        """Start of the timed region: later samples are the ones reported."""
        self._mark = len(self.rows)

    def _read(self):
        for line in self._proc.stdout:
            self.rows.append([c.strip() for c in line.split(",")])

    def stop(self):
        if self._proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self._proc.terminate()
        try:
            self._proc.wait(timeout=5)
        except Exception:
            self._proc.kill()
        if self._thread:
            self._thread.join(timeout=2)
        marked = self.rows[getattr(self, "_mark", 0):]
        rows = marked or self.rows
        sm = [float(r[1]) for r in rows if len(r) >= 9 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if len(r) >= 9 and r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in rows:
            if len(r) >= 9:
                for k, nm in enumerate(names):
                    if r[5 + k].lower() == "active":
                        reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm), "interval_ms": 10,
                "samples_are": "timed region" if marked else "warm-up and timed region (none inside the timed region)"}


def algorithmic_bytes(n_half: int):
    """Algorithmic HBM bytes per atom-step of the mixed path (credited
    independently of the implementation): FP64 positions and velocities read
    and written (48 + 48), F' written and read (8), a half neighbour list read
    by the density and the force pass (2 x 4 n_half), the rebuild amortised
    over 10 steps ((4 n_half + 96) / 10).  Split per kernel: density = list +
    F' write; force = positions + velocities + F' read + list."""
    density = 4 * n_half + 4
    force = 48 + 48 + 4 + 4 * n_half
    rebuild = (4 * n_half + 96) / 10.0
    return {"density": density, "force": force, "rebuild_amortised": rebuild,
            "total": density + force + rebuild}


def run_ours(args):
    import numpy as np
    import torch

    from paper_2405_07898_gb300 import binding, inputs as I

    rank, world, local = _dist()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if args.cells:
        system = I.thermal_system(I.BCC_TA_LIKE, tuple(args.cells), 0.02, 300.0, I.SEED_BASE + 3,
                                  label="bcc_%dx%dx%d" % tuple(args.cells))
    else:
        system = I.bcc_799496()
    n = system.n
    md = binding.MD(system, precision=args.precision, rebuild_every=10, use_graphs=not args.eager,
                    half_list=args.half_list)
    stream = md.stream

    def bench_step():
        md.step(MD_STEPS_PER_BENCH_STEP, DT_FS)

    for _ in range(args.warmup):
        bench_step()
    md.sync()
    launches0 = md.stats()["kernel_launches"]
    clocks = ClockSampler(local)
    clocks.start()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    if args.profiler_range:
        torch.cuda.profiler.start()
    clocks.mark()
    e0.record(stream)
    for _ in range(args.steps):
        bench_step()
    e1.record(stream)
    md.sync()
    if args.profiler_range:
        torch.cuda.profiler.stop()
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms_total = e0.elapsed_time(e1)
    if world > 1:
        from paper_2405_07898_gb300 import sharding
        ms_total = sharding.reduce_max(ms_total, device="cuda")
        torch.distributed.barrier()
    launches = md.stats()["kernel_launches"] - launches0
    ms_per_step = ms_total / args.steps
    ts_per_s = world * args.steps * MD_STEPS_PER_BENCH_STEP / (ms_total * 1e-3)

    # per-kernel durations with CUDA events (eager launches, same kernels)
    prof = md.profile(args.profile_steps, DT_FS)
    st = md.stats()
    n_half = 13  # BCC, r_list = 4.8 A: 26 list entries per atom, 13 per pair direction
    ab = algorithmic_bytes(n_half)
    peak, peak_kind = peaks()
    force_bytes = ab["force"] * n
    achieved = force_bytes / (prof["force_ms"] * 1e-3) / 1e9
    # the recorded capture is of the mixed-precision 799,496-atom force kernel
    traffic = load_traffic() if (args.precision == "mixed" and not args.cells) else None

    # end-to-end through the C ABI with host buffers
    pos_h = torch.from_numpy(system.pos.copy()).pin_memory()
    vel_h = torch.from_numpy(system.vel.copy()).pin_memory()
    md.set_state(pos_h, vel_h, 0)
    md.step(MD_STEPS_PER_BENCH_STEP, DT_FS)
    md.energy()
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        md.set_state(pos_h, vel_h, 0)
        md.step(MD_STEPS_PER_BENCH_STEP, DT_FS)
        md.energy()
    e2e_s = time.perf_counter() - t0
    e2e_value = world * args.e2e_steps * MD_STEPS_PER_BENCH_STEP / e2e_s
    md.close()

    extras = {}
    if rank == 0 and world == 1 and not args.no_extras and not args.cells:
        extras = extra_legs(args, system, ts_per_s)
    if rank == 0:
        cpu = cpu_baseline(args) if (world == 1 and not args.no_cpu_baseline) else None
        line = {
            "metric": f"timesteps/s at 800k atoms ({'mixed precision' if args.precision == 'mixed' else 'FP64'} EAM MD)",
            "value": ts_per_s,
            "unit": "timesteps/s",
            "n_gpus": world,
            "steps": args.steps,
            "warmup": args.warmup,
            "ms_per_step": ms_per_step,
            "higher_is_better": True,
            "scaling": "weak",
            "vs_baseline": None,
            "dtype": "f32+f64" if args.precision == "mixed" else "f64",
            "data": "synthetic: seeded BCC lattice, Gaussian displacements, Maxwell velocities",
            "config": {"workload": (WORKLOAD if not args.cells else system.label + "_mixed").replace(
                           "_mixed", "_" + args.precision), "atoms": n, "md_steps_per_step": MD_STEPS_PER_BENCH_STEP,
                       "dt_fs": DT_FS, "rebuild_every": 10, "precision": args.precision,
                       "list": ("half Verlet list (each pair once), r_list 4.8 A, 13 entries/atom" if args.half_list
                                else "full Verlet list, r_list 4.8 A, 26 entries/atom"),
                       "l2": "working set ~0.35 GB > L2 (no flush needed)",
                       "parallelism": "replicas" if world > 1 else "single GPU",
                       "launch": "eager" if args.eager else "cuda graphs",
                       "atom_steps_per_s": ts_per_s * n},
            "e2e": {"value": e2e_value, "unit": "timesteps/s",
                    "h2d_bytes_per_step": 2 * 3 * n * 8, "d2h_bytes_per_step": 16},
            "gpu_launches": int(launches),
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "kernel": "k_force (force + integration)", "peak_kind": peak_kind,
                         "algorithmic_bytes_per_atom": ab["force"],
                         "kernel_ms": prof["force_ms"]},
            "kernels_ms": {"density": prof["density_ms"], "force": prof["force_ms"],
                           "rebuild": prof["rebuild_ms"], "step": prof["step_ms"]},
            "whole_step_hbm_frac": ab["total"] * n * ts_per_s / world / 1e9 / peak,
            "clocks": clk,
            "stats": {"rebuilds": st["rebuilds"], "max_neighbors": st["max_neighbors"],
                      "lanes_density": st["lanes_density"], "lanes_force": st["lanes_force"],
                      "threads_density": st["threads_density"], "threads_force": st["threads_force"]},
        }
        if cpu is not None:
            line["cpu_baseline"] = cpu
        line.update(extras)
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def extra_legs(args, system, mixed_ts_per_s):
    """Short measurements beside the headline, in the same run: the plain
    FP64 GPU path and the half-list form on the same 799,496-atom system
    (device time of whole bench steps, CUDA events on the library's stream),
    the 512-replica batched launch, one force-matching loss and gradient
    (with its agreement with finite differences on 6 knots), and the oracle
    on all host cores."""
    import torch
    from paper_2405_07898_gb300 import binding, inputs as I

    out = {}
    # FP64 GPU path: the comparison the mixed form is held to (>= 1.5x)
    with binding.MD(system, precision="fp64", rebuild_every=10) as md:
        md.step(MD_STEPS_PER_BENCH_STEP, DT_FS)
        k = 3
        t = _timed_steps(md, MD_STEPS_PER_BENCH_STEP, DT_FS, reps=k)
        v = k * MD_STEPS_PER_BENCH_STEP / t
    out["fp64"] = {"value": v, "unit": "timesteps/s", "bench_steps": k,
                   "mixed_over_fp64": mixed_ts_per_s / v,
                   "note": "plain FP64 GPU path (all pair, density and force arithmetic in FP64), same system"}
    # half lists: each pair once, the other end's terms through fixed-point sums
    with binding.MD(system, precision="mixed", rebuild_every=10, half_list=True) as md:
        for _ in range(3):
            md.step(MD_STEPS_PER_BENCH_STEP, DT_FS)
        k = 30
        t = _timed_steps(md, MD_STEPS_PER_BENCH_STEP, DT_FS, reps=k)
        prof = md.profile(args.profile_steps, DT_FS)
        st = md.stats()
    out["half_list"] = {"value": k * MD_STEPS_PER_BENCH_STEP / t, "unit": "timesteps/s", "bench_steps": k,
                        "max_neighbors": st["max_neighbors"],
                        "kernels_ms": {"density": prof["density_ms"], "force": prof["force_ms"],
                                       "rebuild": prof["rebuild_ms"], "step": prof["step_ms"]},
                        "note": "density = pair pass + F' pass; force = pair pass + integration pass"}
    # the batched form: 512 replicas of uneven size in one persistent launch
    reps = I.replica_batch(512)
    with binding.MDBatch(reps) as b:
        b.step(10, DT_FS)
        b.energy()
        info = b.info()
        nsteps = args.batch_steps_extra
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(b.stream)
        b.step(nsteps, DT_FS)
        e1.record(b.stream)
        b.energy()
        ms = e0.elapsed_time(e1)
    out["batch"] = {"value": info["atoms"] * nsteps / (ms * 1e-3), "unit": "atom-steps/s",
                    "workload": "replicas_512_bcc_fcc_mixed", "replicas": info["replicas"], "atoms": info["atoms"],
                    "steps": nsteps, "ms": ms, "threads_per_block": info["threads_per_block"]}
    # the differentiated form: one force-matching loss and its knot gradient
    adj = adjoint_leg(reps=3, n_fd=6)
    out["adjoint"] = {k: v for k, v in adj.items() if k not in ("higher_is_better",)}
    if not args.no_cpu_baseline:
        out["cpu_baseline_all_cores"] = cpu_baseline_all_cores(args)
    return out


def _timed_steps(md, nsteps, dt, reps=1):
    import torch
    md.sync()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(md.stream)
    for _ in range(reps):
        md.step(nsteps, dt)
    e1.record(md.stream)
    md.sync()
    return e0.elapsed_time(e1) * 1e-3


def _oracle_steps(systems, nsteps: int):
    """Seconds the serial FP64 oracle takes for nsteps timesteps of each
    system (list builds included), and the atom-steps done."""
    import oracle as O

    total, atom_steps = 0.0, 0
    for s in systems:
        sysm = O.System(O.Potential(s.pot), s.box, s.pos, s.vel, s.types)
        t0 = time.perf_counter()
        sysm.step(nsteps, DT_FS)
        total += time.perf_counter() - t0
        atom_steps += s.n * nsteps
    return total, atom_steps


def run_sweep(args):
    """Strong-scaling sweep: BCC cubes of 1,024 .. 314,928 atoms and the
    799,496-atom box at 1,000 K (mixed precision): timesteps/s of md_step
    replayed as CUDA graphs, and up to 314,928 atoms as one cooperative launch
    per call (the library takes the single launch automatically up to 65,536
    atoms).  Beside each size, unless --no-cpu-baseline: the serial FP64
    oracle on one host core, 100 timesteps up to 50,000 atoms and 10 above."""
    import torch
    from paper_2405_07898_gb300 import binding, inputs as I

    # the oracle runs before the first GPU call
    systems = I.sweep_systems(temperature=1000.0)
    cpu = {}
    if not args.no_cpu_baseline:
        for s in systems:
            k = 100 if s.n <= 50000 else 10
            t, _ = _oracle_steps([s], k)
            cpu[s.n] = (k, k / t)
    torch.cuda.set_device(0)
    rows = []
    for s in systems:
        steps = max(200, min(20000, int(2e8 // s.n) // 10 * 10))
        row = {"atoms": s.n, "steps": steps}
        for mode in ("off", "on"):
            if mode == "on" and s.n > 400000:
                continue
            md = binding.MD(s, precision="mixed", persistent=mode)
            md.step(100, DT_FS)
            t = _timed_steps(md, steps, DT_FS)
            key = {"off": "graph", "on": "single_launch"}[mode]
            row[key + "_ts_per_s"] = steps / t
            row[key + "_atom_steps_per_s"] = s.n * steps / t
            if mode != "off":
                st = md.stats()
                row[key + "_blocks"] = st["persistent_blocks"]
                row[key + "_lanes"] = st["persistent_lanes"]
            md.close()
        if s.n in cpu:
            row["oracle_steps"], row["oracle_ts_per_s"] = cpu[s.n]
            row["oracle_atom_steps_per_s"] = s.n * cpu[s.n][1]
            row["oracle_cores"] = 1
        rows.append(row)
    print(json.dumps({"workload": "bcc_sweep_1000K_mixed", "unit": "timesteps/s", "sweep": rows}), flush=True)


def run_batch(args):
    """Batched replicas: 512 independent periodic systems of uneven size (half
    BCC, half FCC, 200-1,200 K) advanced --batch-steps steps in one persistent
    launch per md_batch_step call; atom-steps/s = sum of atoms x steps over
    the CUDA-event time on the batch's stream."""
    import torch
    from paper_2405_07898_gb300 import binding, inputs as I

    reps = I.replica_batch(512)
    cpu = None
    if not args.no_cpu_baseline:
        # the oracle on every 32nd replica (8 BCC, 8 FCC), 10 steps each, before
        # the first GPU call; its atom-steps/s stands for the whole batch
        sample = reps[::32]
        t, done = _oracle_steps(sample, 10)
        cpu = {"value": done / t, "unit": "atom-steps/s", "cores": 1, "kind": "oracle",
               "sample": f"10 timesteps of every 32nd replica ({len(sample)} replicas, "
                         f"{sum(x.n for x in sample):,} atoms; serial FP64 C oracle), {t:.1f} s"}
    torch.cuda.set_device(0)
    b = binding.MDBatch(reps)
    b.step(10, DT_FS)
    b.energy()
    info0 = b.info()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    if args.profiler_range:
        torch.cuda.profiler.start()
    e0.record(b.stream)
    b.step(args.batch_steps, DT_FS)
    e1.record(b.stream)
    if args.profiler_range:
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
    b.energy()
    ms = e0.elapsed_time(e1)
    info = b.info()
    b.close()
    line = {"workload": "replicas_512_bcc_fcc_mixed", "metric": "atom-steps/s",
            "value": info["atoms"] * args.batch_steps / (ms * 1e-3), "unit": "atom-steps/s",
            "replicas": info["replicas"], "atoms": info["atoms"], "steps": args.batch_steps,
            "ms": ms, "kernel_launches": info["kernel_launches"] - info0["kernel_launches"],
            "blocks": info["blocks"], "threads_per_block": info["threads_per_block"],
            "rebuilds": info["rebuilds"] - info0["rebuilds"]}
    if cpu is not None:
        line["cpu_baseline"] = cpu
    print(json.dumps(line), flush=True)


def adjoint_leg(reps: int = 3, n_fd: int = 12):
    """Differentiation: force-matching loss over 64 BCC configurations of
    2,000 atoms and its gradient over 3 x 64 spline knots (adjoint kernels,
    FP64): seconds per loss+gradient evaluation, and the relative difference
    of the gradient from central finite differences of the loss on a seeded
    sample of n_fd knots."""
    import numpy as np
    import torch
    from paper_2405_07898_gb300 import autodiff, inputs as I

    torch.cuda.set_device(0)
    prob = I.fit_problem()
    fm = autodiff.ForceMatch(prob)
    theta = prob.theta0.copy()
    fm.evaluate(theta, grad=True)
    t0 = time.perf_counter()
    for _ in range(reps):
        loss, g = fm.evaluate(theta, grad=True)
    t_eval = (time.perf_counter() - t0) / reps
    rng = np.random.default_rng(7898)
    ks = rng.choice(len(theta), size=n_fd, replace=False)
    fd = []
    for k in ks:
        h = 1e-5 * max(abs(theta[k]), 1e-3)
        tp, tm = theta.copy(), theta.copy()
        tp[k] += h
        tm[k] -= h
        fd.append((fm.evaluate(tp, grad=False)[0] - fm.evaluate(tm, grad=False)[0]) / (2 * h))
    fd = np.array(fd)
    err = float(np.linalg.norm(g[ks] - fd) / np.linalg.norm(fd))
    fm.close()
    return {"workload": "force_match_64x2000_bcc", "metric": "s per loss+gradient", "value": t_eval, "unit": "s",
            "higher_is_better": False, "configs": len(prob.configs), "knots": int(len(theta)),
            "loss": float(loss), f"gradient_vs_central_fd_rel_err_{n_fd}_knots": err}


def run_adjoint(args):
    """The differentiation workload as its own JSON line (adjoint_leg)."""
    print(json.dumps(adjoint_leg()), flush=True)


def run_slab(args):
    """The paper's benchmark geometry: open slabs of 801,792 atoms with open
    boundaries on all axes, mixed precision, dt = 2 fs -- the tantalum size
    (256 x 261 x 6 BCC cells, BCC stand-in potential, 14 interactions per
    atom) and the copper size (174 x 192 x 6 FCC cells, FCC stand-in, 42
    interactions): timesteps/s of md_step (CUDA events on the library's
    stream) and the per-kernel durations."""
    import torch
    from paper_2405_07898_gb300 import binding, inputs as I

    torch.cuda.set_device(0)
    runs = []
    for make in (I.ta_slab_801792, I.cu_slab_801792):
        s = make()
        with binding.MD(s, precision="mixed") as md:
            md.step(50, DT_FS)
            steps = 300
            t = _timed_steps(md, steps, DT_FS)
            prof = md.profile(args.profile_steps, DT_FS)
            st = md.stats()
        runs.append({"system": s.label, "atoms": s.n, "open_axes": s.open_axes, "steps": steps,
                     "ts_per_s": steps / t, "atom_steps_per_s": s.n * steps / t,
                     "kernels_ms": {"density": prof["density_ms"], "force": prof["force_ms"],
                                    "rebuild": prof["rebuild_ms"]},
                     "max_neighbors": st["max_neighbors"], "rebuilds": st["rebuilds"],
                     "lanes": [st["lanes_density"], st["lanes_force"]]})
    print(json.dumps({"workload": "open_slabs_801792_mixed", "metric": "timesteps/s", "unit": "timesteps/s",
                      "runs": runs}), flush=True)


def run_model(args):
    """GB300 counterpart of the paper's linear time model (Eq. 6), which
    writes the time of a timestep as a cost per candidate, a cost per
    interaction and a fixed cost.  The 799,496-atom BCC system is evaluated
    at dt = 0 (nothing moves) for cutoffs and skins that vary the list length
    n_list (entries per atom, within r_cut + skin) and the interactions
    n_inter (within r_cut) independently; the list is rebuilt every step so
    that each evaluation also times a build over n_cand = 27 cells' atoms.
    Least-squares fits, in ns per atom:
      density + force = a n_list + b n_inter + c
      list build      = a' n_cand + b' n_list + c'."""
    import dataclasses

    import numpy as np
    import torch
    from paper_2405_07898_gb300 import binding, inputs as I

    torch.cuda.set_device(0)
    grid = [(3.5, 0.3), (3.5, 0.8), (3.5, 1.4), (4.5, 0.3), (4.5, 0.7), (4.5, 1.1), (5.0, 0.3), (5.0, 0.9),
            (5.6, 0.3), (5.6, 0.9), (6.2, 0.3), (6.2, 0.9)]
    rng = np.random.default_rng(7898)
    rows = []
    for r_cut, skin in grid:
        p = dataclasses.replace(I.BCC_TA_LIKE, r_cut=r_cut, skin=skin)
        s = I.thermal_system(p, (74, 74, 73), 0.02, 300.0, I.SEED_BASE + 1, label="bcc_799496")
        with binding.MD(s, precision="mixed", persistent="off", rebuild_every=1) as md:
            prof = md.profile(args.profile_steps, 0.0)
            off, js = md.neighbors()
            pos, _, _ = md.get_state()
            nc, _, _ = md.cells()
        n = s.n
        n_list = off[-1] / n
        sample = rng.choice(n, size=4000, replace=False)
        inter = 0
        for i in sample:
            d = pos[js[off[i]:off[i + 1]]] - pos[i]
            d -= s.box * np.round(d / s.box)
            inter += int(((d * d).sum(1) < r_cut * r_cut).sum())
        n_inter = inter / len(sample)
        n_cand = 27.0 * n / float(np.prod(nc.astype(np.float64)))
        rows.append({"r_cut": r_cut, "skin": skin, "n_list": n_list, "n_inter": n_inter, "n_cand": n_cand,
                     "pair_ns_per_atom": 1e6 * (prof["density_ms"] + prof["force_ms"]) / n,
                     "density_ns_per_atom": 1e6 * prof["density_ms"] / n,
                     "force_ns_per_atom": 1e6 * prof["force_ms"] / n,
                     "build_ns_per_atom": 1e6 * prof["rebuild_ms"] / n})
    from paper_2405_07898_gb300 import timemodel
    fits = timemodel.fit_points(rows)
    print(json.dumps({"workload": "linear_time_model_bcc_799496_mixed", "unit": "ns per atom",
                      "points": rows, **fits}), flush=True)


def run_drift(args):
    """NVE energy drift: the 250,000-atom Sigma-5 bicrystal at 1,000 K and the
    799,496-atom box at 300 K, mixed precision, dt = 2 fs; total energy
    sampled every 100 steps; drift = least-squares slope per atom scaled to
    1e5 steps."""
    import numpy as np
    import torch
    from paper_2405_07898_gb300 import binding, inputs as I

    torch.cuda.set_device(0)
    out = []
    cases = [(I.sigma5_bicrystal(temperature=1000.0), args.drift_steps),
             (I.bcc_799496(), max(args.drift_steps // 10, 1000))]
    for s, nsteps in cases:
        for precision in ("mixed",) if s.n > 300000 else ("mixed", "fp64"):
            if precision == "fp64" and nsteps > 20000:
                nsteps_p = 20000
            else:
                nsteps_p = nsteps
            md = binding.MD(s, precision=precision)
            e = [sum(md.energy())]
            t0 = time.perf_counter()
            for _ in range(nsteps_p // 100):
                md.step(100, DT_FS)
                e.append(sum(md.energy()))
            wall = time.perf_counter() - t0
            e = np.array(e) / s.n
            steps = np.arange(len(e)) * 100.0
            slope = np.polyfit(steps, e, 1)[0]
            out.append({"system": s.label, "atoms": s.n, "precision": precision, "steps": nsteps_p,
                        "drift_ev_per_atom_per_1e5_steps": float(slope * 1e5),
                        "max_abs_dev_ev_per_atom": float(np.abs(e - e[0]).max()),
                        "ts_per_s_with_sampling": nsteps_p / wall})
            md.close()
    print(json.dumps({"workload": "nve_drift", "runs": out}), flush=True)


TRAFFIC_SOURCES = ("pair_kernels.cuh", "device_common.cuh", "md_internal.cuh", "pair_f32.cu")


def kernel_source_sha256():
    """Hash of the sources the force kernel is compiled from."""
    import hashlib
    from paper_2405_07898_gb300 import build
    h = hashlib.sha256()
    for name in TRAFFIC_SOURCES:
        with open(os.path.join(build.CSRC, name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def load_traffic():
    """DRAM bytes per force launch from the committed ncu summary, if the
    kernel sources have not changed since it was taken (else null)."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(p) as fh:
            t = json.load(fh)
        if t.get("source_sha256") != kernel_source_sha256():
            return None
        return t.get("force_dram_bytes_per_launch")
    except (OSError, ValueError):
        return None


def _oracle_sample(nsteps: int):
    import oracle as O
    from paper_2405_07898_gb300 import inputs as I

    s = I.bcc_799496()
    pot = O.Potential(s.pot)
    sysm = O.System(pot, s.box, s.pos, s.vel, s.types)
    t0 = time.perf_counter()
    sysm.step(nsteps, DT_FS)
    dt = time.perf_counter() - t0
    return dt, s.n


def cpu_baseline_all_cores(args):
    """The oracle's OpenMP build (its per-atom loops in parallel; the list
    build serial) on every host core, over the same bounded sample."""
    import oracle as O
    from paper_2405_07898_gb300 import inputs as I

    s = I.bcc_799496()
    pot = O.Potential(s.pot, L=O.lib_omp())
    sysm = O.System(pot, s.box, s.pos, s.vel, s.types)
    steps = args.cpu_steps
    t0 = time.perf_counter()
    sysm.step(steps, DT_FS)
    dt = time.perf_counter() - t0
    cores = os.cpu_count()
    return {"value": steps / dt, "unit": "timesteps/s", "cores": cores, "kind": "oracle",
            "sample": f"{steps} timesteps of the 799,496-atom system (the oracle's OpenMP build on {cores} "
                      f"threads; list build serial), {dt:.1f} s"}


def cpu_baseline(args):
    steps = args.cpu_steps
    dt, n = _oracle_sample(steps)
    return {"value": steps / dt, "unit": "timesteps/s", "cores": 1, "kind": "oracle",
            "sample": f"{steps} timesteps of the 799,496-atom system (serial FP64 C oracle, "
                      f"list rebuilt every 10 steps), {dt:.1f} s"}


def run_reference(args):
    rank, world, _ = _dist()
    if rank != 0:
        return
    import oracle as O
    from paper_2405_07898_gb300 import inputs as I

    s = I.bcc_799496()
    pot = O.Potential(s.pot)
    sysm = O.System(pot, s.box, s.pos, s.vel, s.types)
    # a bounded sample: at most 3 warm-up steps, then the K timed steps or as
    # many of them (at least 3) as fit in about 90 s of the serial oracle
    warm = min(args.warmup, 3)
    for _ in range(warm):
        sysm.step(1, DT_FS)
    nsteps = 0
    t0 = time.perf_counter()
    while nsteps < max(args.steps, 1):
        sysm.step(1, DT_FS)
        nsteps += 1
        if nsteps >= 3 and time.perf_counter() - t0 > 90.0:
            break
    dt = time.perf_counter() - t0
    value = nsteps / dt
    line = {
        "impl": "reference",
        "metric": "timesteps/s at 800k atoms (mixed precision EAM MD)",
        "value": value, "unit": "timesteps/s", "n_gpus": world, "steps": nsteps,
        "warmup": warm, "ms_per_step": dt / nsteps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic: seeded BCC lattice, Gaussian displacements, Maxwell velocities",
        "config": {"workload": WORKLOAD, "atoms": s.n, "md_steps_per_step": 1, "dt_fs": DT_FS,
                   "rebuild_every": 10},
        "cpu_baseline": {"value": value, "unit": "timesteps/s", "cores": 1, "kind": "oracle",
                         "sample": f"{nsteps} of the {args.steps} requested timesteps (capped at ~90 s) after "
                                   f"{warm} warm-up, serial FP64 C oracle, 799,496 atoms"},
        "e2e": {"value": value, "unit": "timesteps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--profile-steps", type=int, default=20)
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--cpu-steps", type=int, default=10)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="leave out the FP64, half-list, batch, adjoint and all-cores legs of the default line")
    ap.add_argument("--batch-steps-extra", type=int, default=200,
                    help="steps of the batch leg in the default line")
    ap.add_argument("--half-list", action="store_true",
                    help="run the timed workload in the half-list form (profiling)")
    ap.add_argument("--workload", default="bcc_799496", choices=["bcc_799496", "sweep", "drift", "batch", "adjoint", "model", "slab"],
                    help="bcc_799496: the benchmark line; sweep / drift: the strong-scaling sweep and the "
                         "NVE drift runs (their own JSON lines)")
    ap.add_argument("--drift-steps", type=int, default=100000)
    ap.add_argument("--batch-steps", type=int, default=1000)
    ap.add_argument("--cells", type=int, nargs=3, default=None,
                    help="BCC cells per axis of a smaller profiling case (default: the 74x74x73 workload)")
    ap.add_argument("--profiler-range", action="store_true",
                    help="bracket the timed steps with cudaProfilerStart/Stop (for ncu --profile-from-start off)")
    ap.add_argument("--eager", action="store_true",
                    help="launch the step kernels one by one instead of replaying CUDA graphs "
                         "(same kernels; lets a profiler list every launch)")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "sweep":
        run_sweep(args)
    elif args.workload == "drift":
        run_drift(args)
    elif args.workload == "batch":
        run_batch(args)
    elif args.workload == "adjoint":
        run_adjoint(args)
    elif args.workload == "model":
        run_model(args)
    elif args.workload == "slab":
        run_slab(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
