"""Benchmark of the SPH hot path on GB300: KDK steps, learned h + batched vs plain.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload headline|sedov|clustered|boxes|sedov-bins|gravity]

One step = one pass of the whole hot path over the particle set: kick, drift,
cell binning (wrap, key, radix sort, permute, adaptive refinement and neighbour
lists), density with the smoothing-length iteration, force, kick, and the global
reductions (CFL dt, conserved sums).

Default (headline) workload: 512 independent periodic boxes of uneven occupancy
(N log-uniform in [1e3, 2e5], 17.45 M particles, each a uniform background plus
Plummer spheres) on adaptive cells.  value = the learned-h + batched form (all
boxes in one context, graph-replayed steps, h iteration from a learned guess
trained before the timed region); beside it the batched form without the guess
and the unbatched plain form (one context and host-driven steps per box), from
the same state at the same h tolerance; inputs resident in HBM.

Prints ONE JSON line (rank 0).  value = particles advanced per second over all
ranks; the device time is taken with CUDA events on the library's stream,
bracketed by a barrier and synchronisations, max over ranks.  Under torchrun each
rank steps its own replica (the path does not shard across GPUs here).

--impl reference times the FP64 brute-force oracle on this host's cores on a
bounded sample of the same workload (the oracle is the only other
implementation of this path), extrapolated to particles/s.

Secondary lines: --workload sedov (Sedov-Taylor 128^3 on the uniform grid),
clustered (256^3 clustered halo field), boxes (the batched boxes, optionally with
--hpredict), sedov-bins (individual time-steps), gravity (near-field gravity).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "SPH step particles/s & pair interactions/s, learned-h+batched vs plain, 1 GB300"
UNIT = "particles/s"
# Algorithmic FP32 operations per accepted pair (FMA = 2, add/mul/div/rsqrt = 1,
# Kahan compensation included; rejected distance tests are NOT counted).
FLOP_DENSITY_PAIR = 69
FLOP_FORCE_PAIR = 86
CPU_SAMPLE_S = 10.0  # least CPU time of the oracle sample behind cpu_baseline
L2_BYTES = 129e6


def _env_rank():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def _max_over_ranks(x: float, dist=None, device: str = "cuda") -> float:
    """The largest of every rank's x (a time): the job ends with its slowest rank."""
    if not dist:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _throughput(world: int, n: int, steps: int, seconds: float) -> float:
    """Whole-job particles per second: every rank advances its own n particles."""
    return world * n * steps / seconds


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except OSError:
        return {}


def fp32_nominal_tflops(sms: int, peaks: dict) -> tuple[float, str]:
    """Nominal plain FP32 ALU peak: SMs x 128 lanes x 2 FLOP (FMA) x max SM clock."""
    mhz = float(peaks.get("sm_max_mhz", 2070.0))
    return sms * 128 * 2 * mhz * 1e6 / 1e12, f"{sms} SMs x 128 FP32 lanes x 2 x {mhz:.0f} MHz"


_FP32_PEAK = None


def fp32_peak_tflops(sms: int, peaks: dict, stream=None) -> tuple[float, str]:
    """Measured plain FP32 FMA throughput of this GPU (sph_fp32_peak: independent FMA
    recurrences, 8 blocks of 256 threads per SM, fastest of 5 launches), with the SM
    clock sampled while it ran; the nominal figure is quoted beside it."""
    global _FP32_PEAK
    if _FP32_PEAK is None:
        import torch
        from paper_1508_00115_gb300 import binding
        dev = torch.cuda.current_device()
        sampler = ClockSampler(_gpu_id(dev))
        sampler.start()
        time.sleep(0.3)
        tf, ms = 0.0, 0.0
        for _ in range(5):  # about a second of FMAs, so that the clock samples see it
            t, m = binding.sph_fp32_peak(stream, iters=1 << 16, reps=5)
            if t > tf:
                tf, ms = t, m
        clk = sampler.stop()
        nom, how = fp32_nominal_tflops(sms, peaks)
        _FP32_PEAK = (tf, f"measured: FFMA probe (sph_fp32_peak) {tf:.1f} TFLOP/s, {ms:.2f} ms per launch, "
                          f"SM clock median {clk.get('sm_mhz')} MHz under it; nominal {nom:.1f} ({how})")
    return _FP32_PEAK


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples while the timed region runs."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    NAMES = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")

    def __init__(self, gpu_id: str):
        self.gpu_id = gpu_id
        self.lines: list[str] = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", self.gpu_id, f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, mx, pw, reasons = [], [], [], set()
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
                pw.append(float(f[2]))
            except ValueError:
                continue
            for name, v in zip(self.NAMES, f[4:8]):
                if v.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "power_w_max": max(pw) if pw else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def _gpu_id(dev: int) -> str:
    import torch
    try:
        u = str(torch.cuda.get_device_properties(dev).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        vis = os.environ.get("CUDA_VISIBLE_DEVICES")
        return vis.split(",")[dev] if vis else str(dev)


def _traffic(kernel: str, summary: str | None = None):
    """Per-launch DRAM bytes of `kernel` from the committed ncu summary, if it was
    taken on the current sources of that kernel (else None)."""
    from paper_1508_00115_gb300 import build as b
    path = os.path.join(ROOT, "profiles", summary or f"{kernel}_sedov128.md")
    digest = b.gravity_kernel_digest() if kernel == "gravity" else b.pair_kernel_digest()
    try:
        text = open(path).read()
    except OSError:
        return None
    src = None
    val = None
    for line in text.splitlines():
        if line.startswith("kernel_digest:"):
            src = line.split(":", 1)[1].split()[0]
        if line.startswith("dram_bytes_per_launch:"):
            val = float(line.split(":", 1)[1].split()[0])
    if src is None or val is None or src != digest:
        return None
    return val


def _schedule(args, binding) -> dict:
    """Tile width / cell factor: fixed when given, else chosen by the autotuner."""
    sweep = binding.SPH_FLAG_AXIS_SWEEP if getattr(args, "axis_sweep", False) else 0
    if args.tile_width == 0 and args.cell_factor == 0:
        return {"flags": binding.SPH_FLAG_AUTOTUNE | sweep}
    return {"flags": sweep, "tile_width": args.tile_width or 16, "cell_factor": args.cell_factor or 1.1}


def workload(seed: int = 2):
    from paper_1508_00115_gb300 import inputs
    return inputs.sedov(128, seed=seed)


def clustered_workload(n_side: int = 256, seed: int = 77):
    """Clustered halo field: n_side^3 particles, 70% in 200 Plummer spheres (scale
    radii log-uniform 1e-3..1e-2, halo masses dN/dM ~ M^-1.9), 30% uniform;
    velocities Gaussian with sigma 0.05, u uniform in [0.5, 2]."""
    from paper_1508_00115_gb300 import inputs
    n = n_side ** 3
    d = inputs.random_velocities(inputs.plummer_mix(n, seed=seed), 0.05, seed + 1)
    d["u"] = np.random.default_rng(seed + 2).uniform(0.5, 2.0, n)
    return d


def boxes_sizes(n_boxes: int = 512, seed: int = 91) -> np.ndarray:
    """Particle counts of the batched boxes: N log-uniform in [1e3, 2e5]."""
    rng = np.random.default_rng(seed)
    return np.exp(rng.uniform(np.log(1e3), np.log(2e5), n_boxes)).astype(np.int64)


def box_particles(b: int, nb: int, seed: int = 91) -> dict:
    """Box b of the batched set: a uniform-plus-Plummer mix (70% in max(1, N/1000)
    halos), masses 1/N, Gaussian velocities of dispersion 0.05."""
    from paper_1508_00115_gb300 import inputs
    d = inputs.plummer_mix(int(nb), seed=seed + 10 + b, n_halos=max(1, int(nb) // 1000))
    return inputs.random_velocities(d, 0.05, seed + 5000 + b)


def boxes_workload(n_boxes: int = 512, seed: int = 91):
    """Independent periodic unit boxes, N log-uniform in [1e3, 2e5]; each a
    uniform-plus-Plummer mix (70% in max(1, N/1000) halos), masses 1/N per box."""
    from paper_1508_00115_gb300 import inputs
    sizes = boxes_sizes(n_boxes, seed)
    offs = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    d = {k: np.empty(int(offs[-1])) for k in inputs.FIELDS}
    for b, nb in enumerate(sizes):
        bd = box_particles(b, int(nb), seed)
        for k in inputs.FIELDS:
            d[k][offs[b]:offs[b + 1]] = bd[k]
    return d, [int(o) for o in offs]


# ------------------------------------------------------------------ CPU oracle


def oracle_sample(d: dict, n_force: int, seed: int = 5, label: str = "Sedov 128^3",
                  local_radius: bool = False, min_seconds: float = 0.0) -> dict:
    """Time the FP64 oracle on a bounded sample of the workload: n_force random
    targets get the full path (h solve + density for them and for every particle
    within 1.5 h of them, then the force sum), each brute-forced against all N.
    particles/s = 1 / (T_density/S_density + T_force/S_force).  local_radius: the
    neighbourhood of a target is 2 x its own h (h spans decades), else 1.5 x max h.
    min_seconds: if the sample took less CPU time than this, it is taken once more
    with n_force scaled up to about that time (at most every particle), and that
    second sample is the one reported."""
    info = _oracle_sample_once(d, n_force, seed, label, local_radius)
    n = d["x"].size
    if info["seconds"] < min_seconds and n_force < n:
        grow = 1.1 * min_seconds / max(info["seconds"], 1e-3)
        info = _oracle_sample_once(d, min(n, int(math.ceil(n_force * grow))), seed, label,
                                   local_radius)
    return info


def _oracle_sample_once(d: dict, n_force: int, seed: int, label: str, local_radius: bool) -> dict:
    import oracle
    n = d["x"].size
    s = oracle.State(**{k: d[k] for k in ("x", "y", "z", "vx", "vy", "vz", "m", "u", "h")})
    rng = np.random.default_rng(seed)
    tf = rng.choice(n, n_force, replace=False)
    R_all = 1.5 * float(np.max(d["h"]))
    near = []
    for i in tf:  # sample selection (not timed): everything that can be a neighbour
        R = 2.0 * float(d["h"][i]) if local_radius else R_all
        dx = s.x - s.x[i]; dx -= np.rint(dx)
        dy = s.y - s.y[i]; dy -= np.rint(dy)
        dz = s.z - s.z[i]; dz -= np.rint(dz)
        near.append(np.nonzero(dx * dx + dy * dy + dz * dz < R * R)[0])
    td = np.unique(np.concatenate([tf] + near))
    t0 = time.perf_counter()
    r = oracle.solve_h(s, targets=td)
    t1 = time.perf_counter()
    h = np.full(n, 1e-30)
    rho = np.ones(n); P = np.zeros(n); c = np.zeros(n); f = np.ones(n); B = np.zeros(n)
    g = oracle.ghost(r["rho"], r["drho_dh"], r["divv"], r["curl_abs"], s.u[td], r["h"])
    h[td] = r["h"]; rho[td] = r["rho"]; P[td] = g["P"]; c[td] = g["c"]; f[td] = g["f"]
    B[td] = g["B"]
    t2 = time.perf_counter()
    oracle.force(s, h, rho, P, c, f, B, targets=tf)
    t3 = time.perf_counter()
    td_s, tf_s = t1 - t0, t3 - t2
    per = td_s / td.size + tf_s / tf.size
    return {"value": 1.0 / per, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
            "sample": (f"{td.size} density/h-solve targets + {tf.size} force targets of the "
                       f"{n}-particle {label} state, each brute-forced against all N "
                       f"(FP64, OpenMP); {td_s:.1f} s + {tf_s:.1f} s"),
            "seconds": td_s + tf_s}


def run_reference(args):
    """The oracle as it stands, timed on this host's cores: each step a bounded sample
    of the workload the default arm runs (the largest of the 512 batched boxes, built
    alone; --workload sedov: the Sedov-Taylor 128^3 particles), extrapolated to
    particles/s."""
    rank, world, _ = _env_rank()
    if world > 1 and rank != 0:
        return
    if args.workload == "sedov":
        d = workload()
        label, local, nf = "Sedov 128^3", False, args.cpu_force_targets
        wl = "sedov-taylor 128^3 jittered lattice (2097152 particles), bounded oracle sample per step"
    else:
        sizes = boxes_sizes(args.n_boxes)
        b = int(np.argmax(sizes))
        d = box_particles(b, int(sizes[b]))
        label, local, nf = f"largest box (N={int(sizes[b])}) of the batched set", True, args.cpu_force_targets // 3
        wl = (f"{args.n_boxes} periodic boxes, N log-uniform in [1e3, 2e5] (uniform + Plummer mix): bounded oracle "
              f"sample of the largest box (N={int(sizes[b])}) per step")
    vals = []
    info = None
    for k in range(args.warmup + args.steps):
        info = oracle_sample(d, n_force=nf, seed=100 + k, label=label, local_radius=local)
        if k >= args.warmup:
            vals.append(info["value"])
    v = float(np.median(vals)) if vals else 0.0
    out = {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": None, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "impl": "reference",
           "config": {"workload": wl, "n_particles": int(d["x"].size)},
           "cpu_baseline": {"value": v, "unit": UNIT, "cores": info["cores"], "kind": "oracle",
                            "sample": info["sample"]},
           "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


# ------------------------------------------------------------------ GPU path


def run_ours(args):
    import torch
    from paper_1508_00115_gb300 import binding

    rank, world, local = _env_rank()
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    binding.lib()
    d = workload()
    n = int(d["x"].size)
    stream = torch.cuda.Stream()
    sched = _schedule(args, binding)
    ctx = binding.Context(n, device=local, stream=stream.cuda_stream,
                          flags=binding.SPH_FLAG_TIMING | sched.pop("flags"), **sched)
    parts = binding.Particles(d)
    torch.cuda.synchronize()
    for _ in range(args.warmup):
        ctx.step(parts)
    # both timed paths start from this state
    snap = {k: v.clone() for k, v in parts.t.items()}
    torch.cuda.synchronize()

    def timed(fn, tag):
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.nvtx.range_push(tag)  # profilers can select the timed launches
        e0.record(stream)
        res = fn()
        e1.record(stream)
        torch.cuda.nvtx.range_pop()
        torch.cuda.synchronize()
        ms_ = _max_over_ranks(e0.elapsed_time(e1), dist)
        return ms_, res

    # plain path: one sph_step call per step (host-driven passes), per-kernel events
    ctx.reset_stats()
    floors = 0

    def plain():
        fl = 0
        for _ in range(args.steps):
            _, cons = ctx.step(parts)
            fl += cons["u_floors"]
        return fl

    ms_plain, floors = timed(plain, "host_steps")
    st = ctx.stats()

    # production path: all K steps from one captured CUDA graph, no host sync between.
    # Same starting state and schedule; a fresh context is prepared (hydro pass, cell
    # plan, graph capture) outside the timed region.
    tuned = {"tile_width": int(st["tile_width"]), "cell_factor": float(st["cell_factor"])}
    for k, v in snap.items():
        parts.t[k].copy_(v)
    ctx.close()
    ctx = binding.Context(n, device=local, stream=stream.cuda_stream,
                          flags=binding.SPH_FLAG_AXIS_SWEEP if args.axis_sweep else 0, **tuned)
    ctx.steps(parts, 0)
    sampler = ClockSampler(_gpu_id(local)) if rank == 0 else None
    if sampler:
        sampler.start()
        time.sleep(0.3)
    ctx.reset_stats()
    ms, (dt_last, cons_g) = timed(lambda: ctx.steps(parts, args.steps), "graph_steps")
    clocks = sampler.stop() if sampler else None
    st_g = ctx.stats()
    sec = ms / 1e3
    value = _throughput(world, n, args.steps, sec)
    pairs = st_g["density_pairs"] + st_g["force_pairs"]

    # roofline of the dominant pair kernel (plain FP32 ALU bound)
    props = torch.cuda.get_device_properties(local)
    peaks = _peaks()
    peak, peak_how = fp32_peak_tflops(props.multi_processor_count, peaks, stream.cuda_stream)
    kernels = {
        "density": (st["t_density_ms"], st["density_pairs"] * FLOP_DENSITY_PAIR,
                    st["density_passes"]),
        "force": (st["t_force_ms"], st["force_pairs"] * FLOP_FORCE_PAIR, st["force_passes"]),
    }
    dom = max(kernels, key=lambda k: kernels[k][0])
    t_ms, flops, launches = kernels[dom]
    achieved = flops / (t_ms / 1e3) / 1e12 if t_ms > 0 else 0.0
    traffic = _traffic(dom)
    roofline = {"bound": "alu", "kernel": f"k_{dom}", "achieved": achieved, "peak": peak,
                "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": traffic,
                "peak_source": peak_how,
                "launches": launches, "avg_launch_ms": t_ms / max(launches, 1),
                "other_kernel": {k: {"ms_total": v[0], "tflops": (v[1] / (v[0] / 1e3) / 1e12
                                                                   if v[0] > 0 else 0)}
                                 for k, v in kernels.items() if k != dom}}

    # end to end through the public C-ABI with host buffers (pinned)
    e2e = None
    if not args.no_e2e:
        sched_h = _schedule(args, binding)
        ctx_h = binding.Context(n, device=local, stream=stream.cuda_stream,
                                flags=sched_h.pop("flags"), **sched_h)
        hp = binding.Particles(d, device="cpu", pin=True)
        for _ in range(max(1, args.warmup)):
            ctx_h.step_host(hp)
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            ctx_h.step_host(hp)
        t_e2e = _max_over_ranks(time.perf_counter() - t0, dist)
        e2e = {"value": _throughput(world, n, args.steps, t_e2e), "unit": UNIT,
               "h2d_bytes_per_step": n * (6 * 8 + 8 * 4),
               "d2h_bytes_per_step": n * (6 * 8 + 14 * 4 + 4)}
        ctx_h.close()

    # the force pass in its two forms on the same state and schedule: gather (each
    # pair from both sides) and symmetric (each unordered pair once)
    forms = {}
    for name, fl in (("gather", 0), ("symmetric", binding.SPH_FLAG_SYMMETRIC)):
        for k, v in snap.items():
            parts.t[k].copy_(v)
        cf_ = binding.Context(n, device=local, stream=stream.cuda_stream,
                              flags=binding.SPH_FLAG_TIMING | fl, **tuned)
        cf_.build_cells(parts)
        cf_.density(parts)
        cf_.force(parts)  # untimed first launch
        cf_.reset_stats()
        for _ in range(5):
            cf_.force(parts)
        sf = cf_.stats()
        forms[name] = {"ms_per_pass": sf["t_force_ms"] / max(sf["force_passes"], 1),
                       "pairs_per_pass": sf["force_pairs"] / max(sf["force_passes"], 1),
                       "candidates_per_pass": sf["force_candidates"] / max(sf["force_passes"], 1)}
        cf_.close()
    for k, v in snap.items():
        parts.t[k].copy_(v)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = oracle_sample(d, n_force=args.cpu_force_targets, min_seconds=CPU_SAMPLE_S)
        cpu.pop("seconds", None)

    work_mb = n * (6 * 8 + 14 * 4 + 4 + 3 * 16 + 4 + 8 + 8 + 16) / 1e6
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
           "path": "graph-replayed steps (sph_steps): one captured KDK step, all boxes per launch",
           "plain": {"value": _throughput(world, n, args.steps, ms_plain / 1e3), "unit": UNIT,
                     "ms_per_step": ms_plain / args.steps,
                     "path": "one sph_step call per step, host-driven density passes"},
           "scaling": "weak", "vs_baseline": None, "dtype": "f32",
           "dtype_detail": "FP32 pair arithmetic with compensated sums; FP64 positions, "
                           "kicks/drifts, wrap and global reductions",
           "data": "synthetic",
           "config": {"workload": "sedov-taylor 128^3 jittered lattice, KDK step: cells + "
                                  "density/h-iteration + force + kicks",
                      "n_particles": n, "n_ngb": 48, "h_tol": float(ctx.params.h_tol),
                      "tile_width": int(st["tile_width"]),
                      "cell_factor": round(float(st["cell_factor"]), 3),
                      "schedule": "autotuned" if args.tile_width == 0 and args.cell_factor == 0
                                  else "fixed",
                      "pruning": "axis sweep + tile box" if st["axis_sweep"] else "tile box",
                      "pruning_chosen_by": "autotuner" if args.tile_width == 0 and args.cell_factor == 0
                                           else "--axis-sweep",
                      "l2": f"inputs larger than L2 (~{work_mb:.0f} MB resident per step > 129 MB)",
                      "parallelism": f"replicas x{world}"},
           "pair_interactions_per_s": world * pairs / sec,
           "per_step": {"graph_density_passes": st_g["density_passes"] / args.steps,
                        "graph_density_pairs": st_g["density_pairs"] / args.steps,
                        "density_pairs": st["density_pairs"] / args.steps,
                        "force_pairs": st["force_pairs"] / args.steps,
                        "density_passes": st["density_passes"] / args.steps,
                        "density_targets": st["density_targets"] / args.steps,
                        "density_candidates": st["density_candidates"] / args.steps,
                        "force_candidates": st["force_candidates"] / args.steps,
                        "rebuilds": st["rebuilds"] / args.steps,
                        "t_density_ms": st["t_density_ms"] / args.steps,
                        "t_force_ms": st["t_force_ms"] / args.steps,
                        "t_build_ms": st["t_build_ms"] / args.steps,
                        "u_floors": floors / args.steps},
           "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
           "force_forms": forms, "force_symmetric_chosen": int(st["force_symmetric"]),
           "gpu_launches": int(st_g["kernel_launches"]), "clocks": clocks}
    ctx.close()
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist:
        dist.destroy_process_group()


# ------------------------------------------------- individual time-steps


def run_bins(args):
    """Individual time-steps on the Sedov-Taylor workload: from one state, advance by
    dt_max = 2^L x the global CFL step with sph_step_bins (each particle on its own
    power-of-two step), without and with the time-step limiter (SPH_FLAG_BIN_LIMITER),
    and with global CFL steps (sph_step, the last one cut to land on dt_max); report
    the times, the particle updates each needed, and their total energies."""
    import torch
    from paper_1508_00115_gb300 import binding

    rank, world, local = _env_rank()
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    binding.lib()
    d = workload()
    n = int(d["x"].size)
    stream = torch.cuda.Stream()
    sched = _schedule(args, binding)
    flags = sched.pop("flags")
    ctx = binding.Context(n, device=local, stream=stream.cuda_stream, flags=flags, **sched)
    parts = binding.Particles(d)
    cons = None
    for _ in range(args.warmup):
        _, cons = ctx.step(parts)
    torch.cuda.synchronize()
    dt0 = cons["dt_next"]
    levels = args.levels
    dt_max = dt0 * 2.0 ** levels
    snap = {k: v.clone() for k, v in parts.t.items()}

    def restore():
        for k, v in snap.items():
            parts.t[k].copy_(v)
        torch.cuda.synchronize()

    def timed(fn, tag):
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.nvtx.range_push(tag)
        e0.record(stream)
        res = fn()
        e1.record(stream)
        torch.cuda.nvtx.range_pop()
        torch.cuda.synchronize()
        return _max_over_ranks(e0.elapsed_time(e1), dist), res

    def global_steps():
        t, k, c, dt = 0.0, 0, None, dt0
        while t < dt_max * (1 - 1e-12):
            dt = min(dt, dt_max - t)
            used, c = ctx.step(parts, dt)
            t += used
            k += 1
            dt = c["dt_next"]
        return k, c

    def binned():
        return ctx.step_bins(parts, dt_max, levels)

    binned()  # untimed first call (allocations)
    restore()
    ms_bins, (cons_b, st_b) = timed(binned, "bin_steps")
    restore()
    ms_glob, (n_glob, cons_g) = timed(global_steps, "global_steps")
    # the same from the same state with the time-step limiter: its own context (the
    # flag is a context parameter), on the warmed-up state
    restore()
    ctx_l = binding.Context(n, device=local, stream=stream.cuda_stream, flags=flags | binding.SPH_FLAG_BIN_LIMITER,
                            **sched)
    ctx_l.build_cells(parts)
    ctx_l.density(parts)
    ctx_l.force(parts)
    torch.cuda.synchronize()
    snap_l = {k: v.clone() for k, v in parts.t.items()}

    def binned_lim():
        return ctx_l.step_bins(parts, dt_max, levels)

    binned_lim()  # untimed first call (allocations)
    for k, v in snap_l.items():
        parts.t[k].copy_(v)
    ms_lim, (cons_l, st_l) = timed(binned_lim, "bin_steps_limiter")
    ctx_l.close()
    e_start = float(np.sum(d["m"] * d["u"]))
    out = {"metric": METRIC, "value": _throughput(world, n, n_glob, ms_bins / 1e3), "unit": UNIT,
           "n_gpus": world, "steps": 1, "warmup": args.warmup, "ms_per_step": ms_bins,
           "higher_is_better": True,
           "path": (f"individual time-steps (sph_step_bins, {levels} levels) over dt_max = 2^{levels} x "
                    "the global CFL step; value = particles x global steps covered / time"),
           "global": {"value": _throughput(world, n, n_glob, ms_glob / 1e3), "unit": UNIT, "ms": ms_glob,
                      "steps": n_glob, "updates": n_glob * n,
                      "path": "sph_step at the global CFL dt to the same time"},
           "speedup": ms_glob / ms_bins,
           "bins": {"levels": levels, "dt_max": dt_max, "substeps": st_b["substeps"],
                    "updates": st_b["updates"], "cfl_over": st_b["cfl_over"],
                    "bin_count": [int(v) for v in st_b["bin_count"][:levels + 1]]},
           "limiter": {"ms": ms_lim, "speedup_vs_global": ms_glob / ms_lim,
                       "levels": binding.SPH_BIN_LIMIT_LEVELS, "substeps": st_l["substeps"],
                       "updates": st_l["updates"], "limited": st_l["limited"], "woken": st_l["woken"],
                       "passes": st_l["limit_sweeps"],
                       "bin_count": [int(v) for v in st_l["bin_count"][:levels + 1]],
                       "path": "sph_step_bins with SPH_FLAG_BIN_LIMITER (Saitoh & Makino 2009, factor 4)"},
           "energy": {"start": e_start, "bins": cons_b["e_tot"], "bins_limiter": cons_l["e_tot"],
                      "global": cons_g["e_tot"]},
           "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": "sedov-taylor 128^3 jittered lattice, individual time-steps",
                      "n_particles": n, "n_ngb": 48, "levels": levels,
                      "parallelism": f"replicas x{world}"}}
    ctx.close()
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist:
        dist.destroy_process_group()


# ------------------------------------------------- gravity near field


FLOP_GRAV_PAIR = 20  # 3 FADD + 3 FFMA (r^2) + rsqrt + FMUL + FADD (phi) + 2 FMUL + 3 FFMA (a); FFMA = 2


def run_gravity(args):
    """Near-field gravity (sph_gravity_p2p, Sec. 3.2, Eq. 3) on the Sedov-Taylor
    128^3 particles and the SPH path's own cell grid (cell side 1.25 x max h): every
    particle against every other particle of its own and the 26 adjacent cells.
    L2 is flushed (a 256 MB write) before every timed launch; each launch is timed
    by CUDA events on the library's stream."""
    import torch
    from paper_1508_00115_gb300 import binding

    rank, world, local = _env_rank()
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    binding.lib()
    d = workload()
    n = int(d["x"].size)
    stream = torch.cuda.Stream()
    ctx = binding.Context(n, device=local, stream=stream.cuda_stream, flags=binding.SPH_FLAG_TIMING,
                          tile_width=args.tile_width or 32, cell_factor=args.cell_factor or 1.25)
    parts = binding.Particles(d)
    ctx.build_cells(parts)
    out = None
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    # Plummer softening: by default 1/25 of the mean interparticle spacing (a common
    # choice in cosmological runs); --eps 0 runs Eq. 3 unsoftened
    eps = args.eps if args.eps >= 0 else (1.0 / n) ** (1.0 / 3.0) / 25.0
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            out = ctx.gravity(1.0, eps, out)
    torch.cuda.synchronize()
    ctx.reset_stats()
    sampler = ClockSampler(_gpu_id(local)) if rank == 0 else None
    if sampler:
        sampler.start()
        time.sleep(0.3)
    ms = 0.0
    for _ in range(args.steps):
        with torch.cuda.stream(stream):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ctx.gravity(1.0, eps, out)
            e1.record(stream)
        torch.cuda.synchronize()
        ms += e0.elapsed_time(e1)
    clocks = sampler.stop() if sampler else None
    ms = _max_over_ranks(ms, dist)
    st = ctx.stats()
    pairs = st["grav_pairs"] / args.steps
    sec = ms / 1e3
    props = torch.cuda.get_device_properties(local)
    peak, peak_how = fp32_peak_tflops(props.multi_processor_count, _peaks(), stream.cuda_stream)
    achieved = pairs * FLOP_GRAV_PAIR * args.steps / sec / 1e12
    res = {"metric": "gravity near-field pair interactions/s (Sec. 3.2 node-node tasks), 1 GB300",
           "value": world * pairs * args.steps / sec, "unit": "pair interactions/s", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
           "particles_per_s": world * n * args.steps / sec,
           "path": "sph_gravity_p2p: one launch per step over all tiles of the uniform grid",
           "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": "Sedov-Taylor 128^3 jittered lattice, near-field gravity on the SPH cell grid",
                      "n_particles": n, "nc": int(st["nc"]), "pairs_per_particle": pairs / n,
                      "tile_width": int(st["tile_width"]), "eps": eps, "l2": "flushed before every launch",
                      "parallelism": f"replicas x{world}"},
           "roofline": {"bound": "alu", "kernel": "k_gravity", "achieved": achieved, "peak": peak,
                        "unit": "TFLOP/s", "frac": achieved / peak,
                        "traffic": _traffic("gravity", "gravity_sedov128.md") if abs(eps - 3.125e-4) < 1e-9
                        and int(st["tile_width"]) == 32 else None, "peak_source": peak_how,
                        "flop_per_pair": FLOP_GRAV_PAIR, "launches": args.steps,
                        "avg_launch_ms": ms / args.steps},
           "gpu_launches": int(st["kernel_launches"]), "clocks": clocks}
    ctx.close()
    if rank == 0:
        print(json.dumps(res), flush=True)
    if dist:
        dist.destroy_process_group()


# ------------------------------------------------- adaptive-cell workloads


def _train_predictor(binding, n_side, local, stream):
    """Learned h guess trained on another seed of the clustered field: two steps at
    h_tol 1e-6 collected, six epochs.  Returns (weights, floats)."""
    import torch
    d = clustered_workload(n_side, seed=5)
    n = d["x"].size
    ctx = binding.Context(n, device=local, stream=stream.cuda_stream, h_tol=1e-6, leaf_max=128, tile_width=32,
                          flags=binding.SPH_FLAG_ADAPTIVE | binding.SPH_FLAG_TREE_H_GUESS)
    parts = binding.Particles(d)
    ctx.step(parts)
    F = torch.zeros((2 * n, 6), dtype=torch.float32, device="cuda")
    T = torch.zeros(2 * n, dtype=torch.float32, device="cuda")
    ctx.hp_collect(F, T, 2 * n)
    ctx.step(parts)
    ctx.step(parts)
    ctx.hp_init(1)
    for ep in range(6):
        ctx.hp_train(F, T, epochs=1, lr=1e-3 if ep < 4 else 3e-4, seed=ep + 1)
    wf = ctx.hp_save()
    ctx.close()
    return wf


def run_adaptive(args):
    """Clustered halo field (--workload clustered) or batched uneven boxes
    (--workload boxes) on adaptive cells.  Headline: graph-replayed steps (sph_steps:
    the tree built with its sizes on the device, a fixed number of density passes);
    the per-kernel times of the roofline come from host-driven steps (sph_step per
    step, timed kernels)."""
    import torch
    from paper_1508_00115_gb300 import binding

    rank, world, local = _env_rank()
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    binding.lib()
    offs = None
    if args.workload == "clustered":
        d = clustered_workload(args.side)
        label = f"clustered halo field {args.side}^3 (200 Plummer spheres + 30% uniform)"
    else:
        d, offs = boxes_workload(args.n_boxes)
        label = (f"{args.n_boxes} periodic boxes, N log-uniform in [1e3, 2e5], uniform + Plummer "
                 f"mix, batched in one context")
    n = int(d["x"].size)
    stream = torch.cuda.Stream()
    base = binding.SPH_FLAG_ADAPTIVE | binding.SPH_FLAG_TREE_H_GUESS
    sched = {}
    if args.tile_width == 0 and args.leaf_max == 0:
        base |= binding.SPH_FLAG_AUTOTUNE
    else:
        sched = {"tile_width": args.tile_width or 32, "leaf_max": args.leaf_max or 128}
    wf = _train_predictor(binding, max(64, args.side // 2), local, stream) if args.hpredict else None

    ctx = binding.Context(n, device=local, stream=stream.cuda_stream, box_offsets=offs,
                          flags=base | binding.SPH_FLAG_TIMING, **sched)
    parts = binding.Particles(d)
    for _ in range(args.warmup):
        ctx.step(parts)
    st0 = ctx.stats()
    tuned = {"tile_width": int(st0["tile_width"]), "leaf_max": int(st0["leaf_max"])}
    snap = {k: v.clone() for k, v in parts.t.items()}
    ctx.close()
    torch.cuda.synchronize()

    def timed(flags, graph):
        for k, v in snap.items():
            parts.t[k].copy_(v)
        c = binding.Context(n, device=local, stream=stream.cuda_stream, box_offsets=offs,
                            flags=flags | (0 if graph else binding.SPH_FLAG_TIMING), **tuned)
        if wf is not None and flags & binding.SPH_FLAG_HPREDICT:
            c.hp_load(*wf)
        # first hydro on the snapshot (and, for graph steps, the capture) outside the
        # timed region
        if graph:
            c.steps(parts, 0)
        else:
            c.step(parts)
        c.reset_stats()
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        sampler = ClockSampler(_gpu_id(local)) if rank == 0 else None
        if sampler:
            sampler.start()
            time.sleep(0.3)
        torch.cuda.nvtx.range_push("graph_steps" if graph else "host_steps")
        e0.record(stream)
        fl = 0
        if graph:
            _, cons = c.steps(parts, args.steps)
            fl = cons["u_floors"]
        else:
            for _ in range(args.steps):
                _, cons = c.step(parts)
                fl += cons["u_floors"]
        e1.record(stream)
        torch.cuda.nvtx.range_pop()
        torch.cuda.synchronize()
        clocks = sampler.stop() if sampler else None
        ms_ = _max_over_ranks(e0.elapsed_time(e1), dist)
        st = c.stats()
        c.close()
        return ms_, st, clocks, fl

    base_t = binding.SPH_FLAG_ADAPTIVE
    hp_t = binding.SPH_FLAG_HPREDICT if args.hpredict else 0
    # host-driven steps: per-kernel times for the roofline
    ms_host, st, _, _ = timed(base_t | hp_t, graph=False)
    # graph-replayed steps: the headline (and, with the learned guess, the plain one)
    ms, st_g, clocks, floors = timed(base_t | hp_t, graph=True)
    learned = None
    if args.hpredict:
        ms_plain, st_plain, _, _ = timed(base_t, graph=True)
        # the predictor's effect on the h iteration (host-driven steps iterate to
        # convergence, so their passes and re-run targets show it)
        ms_hp0, st_hp0, _, _ = timed(base_t, graph=False)
        learned = {k: {"density_passes_per_step": s_["density_passes"] / args.steps,
                       "targets_per_particle_per_step": s_["density_targets"] / (args.steps * n),
                       "ms_per_step": m_ / args.steps}
                   for k, (m_, s_) in (("plain", (ms_hp0, st_hp0)), ("learned", (ms_host, st)))}
    else:
        ms_plain, st_plain = ms, st_g
    sec = ms / 1e3
    value = _throughput(world, n, args.steps, sec)
    pairs = st_g["density_pairs"] + st_g["force_pairs"]

    props = torch.cuda.get_device_properties(local)
    peak, peak_how = fp32_peak_tflops(props.multi_processor_count, _peaks(), stream.cuda_stream)
    kernels = {"density": (st["t_density_ms"], st["density_pairs"] * FLOP_DENSITY_PAIR, st["density_passes"]),
               "force": (st["t_force_ms"], st["force_pairs"] * FLOP_FORCE_PAIR, st["force_passes"])}
    dom = max(kernels, key=lambda k: kernels[k][0])
    t_ms, flops, launches = kernels[dom]
    achieved = flops / (t_ms / 1e3) / 1e12 if t_ms > 0 else 0.0
    # DRAM bytes per launch: the batched boxes from the committed summary of the same
    # kernel on a smaller set of them, scaled by the units of work (no summary is kept
    # for the clustered field)
    traffic = _boxes_traffic(dom, launches, st, n) if offs is not None else None
    roofline = {"bound": "alu", "kernel": f"k_{dom} (list mode)", "achieved": achieved, "peak": peak,
                "unit": "TFLOP/s", "frac": achieved / peak, "traffic": traffic,
                "peak_source": peak_how,
                "launches": launches, "avg_launch_ms": t_ms / max(launches, 1)}

    e2e = None
    if not args.no_e2e:
        ctx_h = binding.Context(n, device=local, stream=stream.cuda_stream, box_offsets=offs,
                                flags=base | (binding.SPH_FLAG_HPREDICT if args.hpredict else 0), **tuned)
        if args.hpredict:
            ctx_h.hp_load(*wf)
        hp = binding.Particles({k: snap[k].cpu().numpy() for k in snap}, device="cpu", pin=True)
        ctx_h.step_host(hp)
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            ctx_h.step_host(hp)
        t_e2e = _max_over_ranks(time.perf_counter() - t0, dist)
        e2e = {"value": _throughput(world, n, args.steps, t_e2e), "unit": UNIT,
               "h2d_bytes_per_step": n * (6 * 8 + 8 * 4), "d2h_bytes_per_step": n * (6 * 8 + 14 * 4 + 4)}
        ctx_h.close()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        g = {k: snap[k].cpu().numpy().astype(np.float64) for k in ("x", "y", "z", "vx", "vy", "vz", "m", "u",
                                                                    "h")}
        if offs is not None:  # the largest box, on its own
            b = int(np.argmax(np.diff(offs)))
            g = {k: v[offs[b]:offs[b + 1]] for k, v in g.items()}
            lab = f"largest box (N={offs[b + 1] - offs[b]}) of the batched set"
        else:
            lab = label
        cpu = oracle_sample(g, n_force=args.cpu_force_targets // 3, label=lab, local_radius=True,
                            min_seconds=CPU_SAMPLE_S)
        cpu.pop("seconds", None)

    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
           "path": ("graph-replayed steps (sph_steps) on adaptive cells, tree sizes on the device"
                    + (", learned h guess" if args.hpredict else "")),
           "plain": {"value": _throughput(world, n, args.steps, ms_plain / 1e3), "unit": UNIT,
                     "ms_per_step": ms_plain / args.steps,
                     "density_passes_per_step": st_plain["density_passes"] / args.steps,
                     "path": "graph-replayed steps, h iteration from the previous h"},
           "host_steps": {"value": _throughput(world, n, args.steps, ms_host / 1e3), "unit": UNIT,
                          "ms_per_step": ms_host / args.steps,
                          "density_passes_per_step": st["density_passes"] / args.steps,
                          "rebuilds_per_step": st["rebuilds"] / args.steps,
                          "path": "sph_step per step (host-driven passes, timed kernels)"},
           "scaling": "weak", "vs_baseline": None, "dtype": "f32",
           "dtype_detail": "FP32 pair arithmetic on leaf-relative positions with compensated sums; "
                           "FP64 positions, kicks/drifts, wrap and global reductions; BF16/FP32 MLP",
           "data": "synthetic",
           "config": {"workload": label, "n_particles": n, "n_boxes": len(offs) - 1 if offs else 1,
                      "n_ngb": 48, "h_tol": 1e-4, "tile_width": tuned["tile_width"],
                      "leaf_max": tuned["leaf_max"],
                      "schedule": "autotuned" if not sched else "fixed",
                      "h_guess": "tree density estimate on the first build; learned MLP guess per step"
                                 if args.hpredict else "tree density estimate on the first build",
                      "l2": "inputs larger than L2", "parallelism": f"replicas x{world}"},
           "pair_interactions_per_s": world * pairs / sec,
           "per_step": {"graph_density_passes": st_g["density_passes"] / args.steps,
                        "graph_density_pairs": st_g["density_pairs"] / args.steps,
                        "graph_leaves": st_g["n_cells"],
                        "density_pairs": st["density_pairs"] / args.steps,
                        "force_pairs": st["force_pairs"] / args.steps,
                        "density_passes": st["density_passes"] / args.steps,
                        "density_targets": st["density_targets"] / args.steps,
                        "density_candidates": st["density_candidates"] / args.steps,
                        "force_candidates": st["force_candidates"] / args.steps,
                        "rebuilds": st["rebuilds"] / args.steps, "leaves": st["n_cells"],
                        "t_density_ms": st["t_density_ms"] / args.steps,
                        "t_force_ms": st["t_force_ms"] / args.steps,
                        "t_build_ms": st["t_build_ms"] / args.steps, "u_floors": floors / args.steps},
           "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
           "gpu_launches": int(st_g["kernel_launches"]), "clocks": clocks}
    if learned:
        out["learned_h"] = learned
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist:
        dist.destroy_process_group()


# ------------------------------------------- the headline: learned h + batched vs plain


def _train_boxes_predictor(binding, n_boxes, local, stream):
    """Learned h guess for the batched boxes, trained before the timed region on
    another realisation of the workload (seed 92, a quarter of the boxes): the
    (features, converged log h ratio) pairs of two steps at h_tol 1e-6, six epochs
    of Adam.  Returns (weights, floats) and a description."""
    import torch
    d, offs = boxes_workload(max(8, n_boxes // 4), seed=92)
    n = int(d["x"].size)
    t0 = time.perf_counter()
    ctx = binding.Context(n, device=local, stream=stream.cuda_stream, box_offsets=offs, h_tol=1e-6, leaf_max=128,
                          tile_width=32, flags=binding.SPH_FLAG_ADAPTIVE | binding.SPH_FLAG_TREE_H_GUESS)
    parts = binding.Particles(d)
    # at h_tol 1e-6 a handful of the ~5 M smoothing lengths may end a step at their
    # last iterate (the step completes); their targets are noise among millions
    ok = (binding.SPH_ERR_NOT_CONVERGED,)
    ctx.step(parts, allow=ok)
    F = torch.zeros((2 * n, 6), dtype=torch.float32, device="cuda")
    T = torch.zeros(2 * n, dtype=torch.float32, device="cuda")
    ctx.hp_collect(F, T, 2 * n)
    ctx.step(parts, allow=ok)
    ctx.step(parts, allow=ok)
    ctx.hp_collect(None, None, 0)
    ctx.hp_init(1)
    loss = None
    for ep in range(6):
        loss = ctx.hp_train(F, T, epochs=1, lr=1e-3 if ep < 4 else 3e-4, seed=ep + 1)
    wf = ctx.hp_save()
    ctx.close()
    del F, T, parts
    torch.cuda.empty_cache()
    return wf, {"trained_on": f"{len(offs) - 1} boxes of seed 92 ({n} particles), two steps at h_tol 1e-6",
                "samples": 2 * n, "epochs": 6, "final_loss": loss, "seconds": time.perf_counter() - t0}


def run_headline(args):
    """The metric on the largest single-GPU configuration: 512 independent periodic
    boxes of uneven occupancy (N log-uniform in [1e3, 2e5], clustered: Plummer
    spheres in a uniform background; 17.45 M particles), KDK steps on adaptive cells.

    value   learned h + batched: every box in one context (one persistent launch per
            pass for all boxes), whole steps replayed from a CUDA graph, each step's h
            iteration started from the learned guess (trained before the timed
            region on another realisation).
    plain   the same batched graph without the learned guess (the previous h).
    plain_unbatched  no batching, no learned guess: one context per box, one
            sph_step call per box and step (the box's own launches, host-driven).
    All three start from the same state, at the same h_tol (1e-4); the first two
    alternate over --repeats runs (median reported)."""
    import torch
    from paper_1508_00115_gb300 import binding

    rank, world, local = _env_rank()
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    binding.lib()
    t_setup = time.perf_counter()
    stream = torch.cuda.Stream()
    wf, pred_info = _train_boxes_predictor(binding, args.n_boxes, local, stream)
    d, offs = boxes_workload(args.n_boxes)
    n = int(d["x"].size)
    nb = len(offs) - 1
    base = binding.SPH_FLAG_ADAPTIVE | binding.SPH_FLAG_TREE_H_GUESS
    # warm-up steps on the batched context (the autotuner picks tile width x leaf
    # size on the first density pass); their end state is every arm's start
    ctx = binding.Context(n, device=local, stream=stream.cuda_stream, box_offsets=offs,
                          flags=base | binding.SPH_FLAG_AUTOTUNE)
    parts = binding.Particles(d)
    for _ in range(args.warmup):
        ctx.step(parts)
    st0 = ctx.stats()
    tuned = {"tile_width": int(st0["tile_width"]), "leaf_max": int(st0["leaf_max"])}
    snap = {k: v.clone() for k, v in parts.t.items()}
    ctx.close()
    torch.cuda.synchronize()
    A = binding.SPH_FLAG_ADAPTIVE

    def restore():
        for k, v in snap.items():
            parts.t[k].copy_(v)

    def run(flags, graph, steps, sample_clocks=False):
        restore()
        c = binding.Context(n, device=local, stream=stream.cuda_stream, box_offsets=offs,
                            flags=flags | (0 if graph else binding.SPH_FLAG_TIMING), **tuned)
        if flags & binding.SPH_FLAG_HPREDICT:
            c.hp_load(*wf)
        # the first hydro pass on the snapshot (and, for replayed steps, the capture)
        # outside the timed region
        if graph:
            c.steps(parts, 0)
        else:
            c.step(parts)
        c.reset_stats()
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        sampler = ClockSampler(_gpu_id(local)) if (sample_clocks and rank == 0) else None
        if sampler:
            sampler.start()
            time.sleep(0.3)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        # named range of the timed region (lets a profiler take just these launches)
        torch.cuda.nvtx.range_push(("headline_learned" if flags & binding.SPH_FLAG_HPREDICT else "headline_plain") +
                                   ("_graph" if graph else "_host"))
        e0.record(stream)
        fl = 0
        if graph:
            _, cons = c.steps(parts, steps)
            fl = cons["u_floors"]
        else:
            for _ in range(steps):
                _, cons = c.step(parts)
                fl += cons["u_floors"]
        e1.record(stream)
        torch.cuda.nvtx.range_pop()
        torch.cuda.synchronize()
        clocks = sampler.stop() if sampler else None
        ms_ = _max_over_ranks(e0.elapsed_time(e1), dist)
        st = c.stats()
        c.close()
        return ms_, st, clocks, fl

    learned_ms, plain_ms = [], []
    st_learned = st_plain = clocks = None
    floors = 0
    for r in range(args.repeats):
        m1, s1, ck, fl = run(A | binding.SPH_FLAG_HPREDICT, True, args.steps, sample_clocks=(r == 0))
        m2, s2, _, _ = run(A, True, args.steps)
        learned_ms.append(m1)
        plain_ms.append(m2)
        if r == 0:
            st_learned, st_plain, clocks, floors = s1, s2, ck, fl
    ms = float(np.median(learned_ms))
    ms_plain = float(np.median(plain_ms))
    sec = ms / 1e3
    value = _throughput(world, n, args.steps, sec)
    pairs = st_learned["density_pairs"] + st_learned["force_pairs"]

    # host-driven steps with timed kernels: the per-kernel times of the roofline and
    # the effect of the guess on the h iteration (passes and re-run targets)
    ms_hl, st_hl, _, _ = run(A | binding.SPH_FLAG_HPREDICT, False, args.steps)
    ms_hp, st_hp, _, _ = run(A, False, args.steps)
    learned = {k: {"density_passes_per_step": s_["density_passes"] / args.steps,
                   "density_targets_per_particle_per_step": s_["density_targets"] / (args.steps * n),
                   "t_density_ms_per_step": s_["t_density_ms"] / args.steps,
                   "ms_per_step": m_ / args.steps}
               for k, (m_, s_) in (("plain", (ms_hp, st_hp)), ("learned", (ms_hl, st_hl)))}

    # plain, unbatched: one context per box, host-driven steps
    unb = None
    if args.unbatched_steps > 0:
        restore()
        snap_np = {k: v.cpu().numpy() for k, v in snap.items()}
        ctxs, bparts = [], []
        for b in range(nb):
            sl = slice(offs[b], offs[b + 1])
            cb = binding.Context(offs[b + 1] - offs[b], device=local, stream=stream.cuda_stream, flags=A, **tuned)
            pb = binding.Particles({k: v[sl] for k, v in snap_np.items()})
            cb.build_cells(pb)
            cb.density(pb)
            cb.force(pb)
            ctxs.append(cb)
            bparts.append(pb)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.unbatched_steps):
            for cb, pb in zip(ctxs, bparts):
                cb.step(pb)
        e1.record(stream)
        torch.cuda.synchronize()
        ms_u = _max_over_ranks(e0.elapsed_time(e1), dist)
        launches_u = sum(c.stats()["kernel_launches"] for c in ctxs)
        for cb in ctxs:
            cb.close()
        del bparts
        unb = {"value": _throughput(world, n, args.unbatched_steps, ms_u / 1e3), "unit": UNIT,
               "ms_per_step": ms_u / args.unbatched_steps, "steps": args.unbatched_steps,
               "kernel_launches_per_step": launches_u / args.unbatched_steps,
               "path": f"{nb} contexts, one sph_step per box and step (host-driven passes), previous-h guess"}

    props = torch.cuda.get_device_properties(local)
    peak, peak_how = fp32_peak_tflops(props.multi_processor_count, _peaks(), stream.cuda_stream)
    kernels = {"density": (st_hl["t_density_ms"], st_hl["density_pairs"] * FLOP_DENSITY_PAIR,
                           st_hl["density_passes"]),
               "force": (st_hl["t_force_ms"], st_hl["force_pairs"] * FLOP_FORCE_PAIR, st_hl["force_passes"])}
    dom = max(kernels, key=lambda k: kernels[k][0])
    t_ms, flops, launches = kernels[dom]
    achieved = flops / (t_ms / 1e3) / 1e12 if t_ms > 0 else 0.0
    roofline = {"bound": "alu", "kernel": f"k_{dom} (list mode)", "achieved": achieved, "peak": peak,
                "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": _boxes_traffic(dom, launches, st_hl, n),
                "peak_source": peak_how, "launches": launches, "avg_launch_ms": t_ms / max(launches, 1),
                "timing": "CUDA events around every launch of host-driven learned-h steps (same state, "
                          "schedule and h_tol as the replayed ones)",
                "other_kernel": {k: {"ms_total": v[0], "tflops": (v[1] / (v[0] / 1e3) / 1e12 if v[0] > 0 else 0)}
                                 for k, v in kernels.items() if k != dom}}

    e2e = None
    if not args.no_e2e:
        restore()
        ctx_h = binding.Context(n, device=local, stream=stream.cuda_stream, box_offsets=offs,
                                flags=A | binding.SPH_FLAG_HPREDICT, **tuned)
        ctx_h.hp_load(*wf)
        hp = binding.Particles({k: snap[k].cpu().numpy() for k in snap}, device="cpu", pin=True)
        ctx_h.step_host(hp)
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            ctx_h.step_host(hp)
        t_e2e = _max_over_ranks(time.perf_counter() - t0, dist)
        e2e = {"value": _throughput(world, n, args.steps, t_e2e), "unit": UNIT,
               "h2d_bytes_per_step": n * (6 * 8 + 8 * 4), "d2h_bytes_per_step": n * (6 * 8 + 14 * 4 + 4),
               "path": "sph_step_host (pinned host buffers, learned h, all boxes batched, host-driven passes)"}
        ctx_h.close()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        b = int(np.argmax(np.diff(offs)))
        g = {k: snap[k][offs[b]:offs[b + 1]].cpu().numpy().astype(np.float64)
             for k in ("x", "y", "z", "vx", "vy", "vz", "m", "u", "h")}
        cpu = oracle_sample(g, n_force=args.cpu_force_targets // 3,
                            label=f"largest box (N={offs[b + 1] - offs[b]}) of the batched set",
                            local_radius=True, min_seconds=CPU_SAMPLE_S)
        cpu.pop("seconds", None)

    spread = lambda v: [float(x) / args.steps for x in v]
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
           "path": "learned h + batched: all boxes in one context, graph-replayed steps (sph_steps), h iteration "
                   "from the learned guess",
           "plain": {"value": _throughput(world, n, args.steps, ms_plain / 1e3), "unit": UNIT,
                     "ms_per_step": ms_plain / args.steps,
                     "path": "batched, graph-replayed, h iteration from the previous h (no learned guess)"},
           "plain_unbatched": unb,
           "ratios": {"learned_batched_vs_plain_batched": ms_plain / ms,
                      "learned_batched_vs_plain_unbatched": (unb["ms_per_step"] / (ms / args.steps)) if unb else None},
           "repeats": {"n": args.repeats, "learned_ms_per_step": spread(learned_ms),
                       "plain_ms_per_step": spread(plain_ms)},
           "learned_h": learned, "predictor": pred_info,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32",
           "dtype_detail": "FP32 pair arithmetic on leaf-relative positions with compensated sums; FP64 positions, "
                           "kicks/drifts, wrap and global reductions; BF16/FP32 MLP",
           "data": "synthetic",
           "config": {"workload": f"{nb} periodic boxes, N log-uniform in [1e3, 2e5] (uniform + Plummer mix), "
                                  "batched, learned h",
                      "n_particles": n, "n_boxes": nb, "n_ngb": 48, "h_tol": 1e-4,
                      "tile_width": tuned["tile_width"], "leaf_max": tuned["leaf_max"], "schedule": "autotuned",
                      "l2": "inputs larger than L2 (~7 GB resident)", "parallelism": f"replicas x{world}"},
           "pair_interactions_per_s": world * pairs / sec,
           "per_step": {"graph_density_passes": st_learned["density_passes"] / args.steps,
                        "graph_density_pairs": st_learned["density_pairs"] / args.steps,
                        "force_pairs": st_learned["force_pairs"] / args.steps,
                        "leaves": st_learned["n_cells"],
                        "density_candidates": st_hl["density_candidates"] / args.steps,
                        "force_candidates": st_hl["force_candidates"] / args.steps,
                        "density_streamed": st_hl["density_streamed"] / args.steps,
                        "density_staged": st_hl["density_staged"] / args.steps,
                        "force_streamed": st_hl["force_streamed"] / args.steps,
                        "force_staged": st_hl["force_staged"] / args.steps,
                        "density_pairs_host": st_hl["density_pairs"] / args.steps,
                        "t_density_ms": st_hl["t_density_ms"] / args.steps,
                        "t_force_ms": st_hl["t_force_ms"] / args.steps,
                        "t_build_ms": st_hl["t_build_ms"] / args.steps, "u_floors": floors / args.steps},
           "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
           "gpu_launches": int(st_learned["kernel_launches"]), "clocks": clocks,
           "setup_s": time.perf_counter() - t_setup}
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist:
        dist.destroy_process_group()


def _boxes_traffic(kernel, launches, st, n):
    """DRAM bytes per launch of the list-mode kernel, scaled to this workload from the
    committed ncu summary of a smaller batched set (profiles/<kernel>_boxes.md: bytes
    per unit of work -- per target for the density, per particle for the force),
    while the pair kernels' sources are those it was taken on; else None."""
    from paper_1508_00115_gb300 import build as b
    path = os.path.join(ROOT, "profiles", f"{kernel}_boxes.md")
    try:
        text = open(path).read()
    except OSError:
        return None
    src = per = None
    for line in text.splitlines():
        if line.startswith("kernel_digest:"):
            src = line.split(":", 1)[1].split()[0]
        if line.startswith("dram_bytes_per_unit:"):
            per = float(line.split(":", 1)[1].split()[0])
    if src is None or per is None or src != b.pair_kernel_digest():
        return None
    units = st["density_targets"] if kernel == "density" else n * launches
    return per * units / max(launches, 1)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-force-targets", type=int, default=48)
    ap.add_argument("--tile-width", type=int, default=0, help="16 or 32 (0: autotuned)")
    ap.add_argument("--cell-factor", type=float, default=0.0, help=">= 1 (0: autotuned)")
    ap.add_argument("--workload", choices=["headline", "sedov", "clustered", "boxes", "sedov-bins", "gravity"],
                    default="headline",
                    help="headline: 512 uneven clustered boxes, learned h + batched against plain (the metric); "
                         "sedov: Sedov-Taylor 128^3 on the uniform grid; clustered: clustered halo field on "
                         "adaptive cells; boxes: batched uneven boxes on adaptive cells; sedov-bins: "
                         "individual time-steps against global steps on the Sedov workload; gravity: near-field "
                         "gravity on the Sedov particles")
    ap.add_argument("--repeats", type=int, default=3, help="headline: alternating learned / plain runs")
    ap.add_argument("--unbatched-steps", type=int, default=2,
                    help="headline: steps of the unbatched plain arm (0: skip it)")
    ap.add_argument("--levels", type=int, default=8, help="sedov-bins: time-bin levels")
    ap.add_argument("--eps", type=float, default=-1.0,
                    help="gravity: Plummer softening (default: 1/25 of the mean spacing; 0: unsoftened)")
    ap.add_argument("--side", type=int, default=256, help="clustered: particles per side")
    ap.add_argument("--n-boxes", type=int, default=512, help="boxes: number of boxes")
    ap.add_argument("--leaf-max", type=int, default=0, help="adaptive: leaf size (0: autotuned)")
    ap.add_argument("--axis-sweep", action="store_true",
                    help="sedov: sort cells along the 13 half-stencil axes and sweep (SPH_FLAG_AXIS_SWEEP)")
    ap.add_argument("--hpredict", action="store_true",
                    help="adaptive workloads: train the learned h guess on another seed and use it")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "sedov-bins":
        run_bins(args)
    elif args.workload == "gravity":
        run_gravity(args)
    elif args.workload == "headline":
        run_headline(args)
    elif args.workload != "sedov":
        run_adaptive(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
