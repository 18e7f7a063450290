"""Benchmark: particle-steps/s of the Kob-Andersen MD step on GB300.

Workload: Kob-Andersen 80:20 mixture (Sec. 5 parameters), N = 65536,
density 1.2, dt = 0.001, truncated-and-shifted at 2.5 sigma_ab, skin 0.3,
mixed precision (FP32 pair forces, double-single positions/velocities and
integration, compensated force summation, FP64 reductions).  Synthetic input:
seeded fcc lattice, melted at T = 2 and quenched to T = 0.5 by velocity
rescaling (4000 steps, untimed), then timed in NVE.

One timed iteration ("step" of this script) = md_step(1000): 1000 MD steps
with every neighbour-list rebuild, reorder and per-step reduction, executed
as one CUDA graph.  The L2 cache is flushed (256 MB write) between timed
iterations; within one the state stays on chip, as in a continuous run.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

With --gpus N > 1 (launched by torch.distributed.run) every rank advances its
own independent replica (no data-path collective): weak scaling, "replicas
only".  --impl reference times the FP64 CPU oracle on the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "particle-steps/s at KA N=65536 (mixed vs FP64 on GB300) at stated energy drift/step"

# Workload constants of the paper's protocols
KA_DT = 0.001                                     # Kob-Andersen time step (Sec. 5)
E1 = {"temperature": 1.5, "dt": 0.001, "skin": 0.5}   # performance measurements (Sec. 3)
STABILITY = {"n": 10000, "density": 0.75, "temperature": 1.12, "dts": (0.001, 0.003),
             "smooth": (0.0, 0.005)}              # stability protocol (Sec. 4)
UNIT = "particle-steps/s"


def parse_args(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--particles", dest="n", type=int, default=65536)
    ap.add_argument("--inner", type=int, default=1000, help="MD steps per timed iteration")
    ap.add_argument("--precision", choices=["mixed", "fp64", "fp32"], default="mixed")
    ap.add_argument("--no-extras", action="store_true", help="skip fp64 / e2e / cpu legs")
    ap.add_argument("--no-graph", action="store_true",
                    help="plain stream launches instead of the CUDA graph (for per-kernel profiling)")
    ap.add_argument("--tpp", type=int, default=0, help="force-kernel threads per particle (0 = auto)")
    ap.add_argument("--step-form", type=int, default=0, choices=[0, 1, 2],
                    help="step-kernel blocks: 0 auto, 1 one per chunk, 2 resident blocks sweep (not FP64)")
    ap.add_argument("--build-form", type=int, default=0, choices=[0, 1, 2],
                    help="neighbour build: 0 auto, 1 one warp per cell, 2 one block per cell")
    ap.add_argument("--check", type=int, default=0,
                    help="MD steps between rebuild checks of the graph (0 = the library's choice)")
    ap.add_argument("--skin", type=float, default=0.3, help="neighbour-list skin (with --no-tune)")
    ap.add_argument("--no-tune", action="store_true", help="skip the autotuner (lanes, skin, capacity)")
    ap.add_argument("--workload", choices=["ka65536", "lj-sweep", "e1", "replicas", "drift", "stability",
                                           "longrun", "stats", "drift-floor"],
                    default="ka65536",
                    help="ka65536: the headline line; the others print one line per case")
    ap.add_argument("--sizes", type=int, nargs="*", default=None, help="lj-sweep / e1 particle counts")
    ap.add_argument("--densities", type=float, nargs="*", default=None, help="e1 number densities")
    ap.add_argument("--md-steps", type=int, default=100000, help="drift: NVE MD steps per run")
    ap.add_argument("--fp64-steps", type=int, default=None,
                    help="longrun: FP64 NVE steps (default a fifth of --md-steps)")
    ap.add_argument("--cases", nargs="*", default=None, help="drift: subset of cases")
    ap.add_argument("--seeds", type=int, nargs="*", default=None,
                    help="stats / longrun: seeds of the independent runs")
    ap.add_argument("--precisions", nargs="*", default=None, help="stats / drift-floor / longrun: precisions")
    ap.add_argument("--dt", type=float, default=None, help="longrun: time step (default 0.001)")
    ap.add_argument("--smooth", type=float, nargs="*", default=None, help="longrun: smoothing widths h")
    return ap.parse_args(argv)


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def aggregate(work_per_rank, seconds_per_rank):
    """Whole-job throughput: all ranks' work over the slowest rank's time."""
    t = max(seconds_per_rank)
    return (sum(work_per_rank) / t if t > 0 else 0.0), t


def allgather_floats(values, world):
    """Gather a list of floats from every rank (identity when world == 1)."""
    if world == 1:
        return [list(values)]
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor(values, dtype=torch.float64, device=dev)
    out = [torch.zeros_like(t) for _ in range(world)]
    dist.all_gather(out, t)
    return [o.cpu().tolist() for o in out]


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if f[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(smax)) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except OSError:
        return None


# Algorithmic arithmetic of the mixed pair loop per entry of a particle's list
# and per pair inside the cutoff (add / mul / rcp / rint = 1, FMA = 2): the
# method's own count for double-single-corrected minimum-image separations
# (26 per entry) and force, energy and virial with compensated accumulation
# (38 per pair).  This is the convention the roofline's `achieved` uses.
FLOP_PER_ENTRY_METHOD = 26
FLOP_PER_PAIR_METHOD = 38
# The plain (FP64 or FP32) count of the same method: separation 20 per entry,
# force, energy and virial 20 per pair, no compensation.
FLOP_PER_ENTRY_PLAIN = 20
FLOP_PER_PAIR_PLAIN = 20
# The same work counted as this kernel does it (reported beside): separation
# from the 32-bit fixed-point positions 3 x (integer difference, conversion,
# scale) = 9, r^2 = 5, cutoff test = 1; inside the cutoff: reciprocal 1,
# (sigma^2/r^2)^3 = 3, force factor 4, three products with the separation 3,
# energy 2 FMA + sum 5, Kahan accumulation 4 x 4.
FLOP_PER_ENTRY = 15
FLOP_PER_PAIR = 32
# per particle and step, the double-single velocity-Verlet update fused into
# the same kernel: two half kicks 3 x 2 x (product 8 + sum 11), drift
# 3 x (product 10 + sum 11 + re-anchor 6), displacement 15
FLOP_PER_UPDATE = 210


KERNEL_SOURCES = ("paper_0912_3824_gb300/csrc/md_kernels.cuh", "paper_0912_3824_gb300/csrc/md_common.cuh")


def profiled_traffic(kernel, skin):
    """DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum)
    of `kernel` from the committed ncu summary, or None when no summary
    covers it, its sources changed since the capture, or the capture ran with
    another skin (another list length)."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "k_step_ka65536_mixed.md")
    if not os.path.exists(path):
        return None
    fields = {}
    for line in open(path):
        k, sep, v = line.partition(":")
        if sep and k in ("traffic_bytes_per_launch", "kernel", "source_sha256", "skin"):
            fields[k] = v.strip()
    now = " ".join(hashlib.sha256(open(os.path.join(ROOT, f), "rb").read()).hexdigest() for f in KERNEL_SOURCES)
    if fields.get("kernel") != kernel or fields.get("source_sha256") != now:
        return None
    if abs(float(fields.get("skin", "nan")) - float(skin)) > 1e-9:
        return None
    return float(fields["traffic_bytes_per_launch"])


def list_statistics(sim, params, sample=100000):
    """Mean list length and mean number of pairs inside the cutoff, from the
    current lists and positions (host-side numpy; at most `sample` particles,
    evenly strided, enter the cutoff count).  Single-box handles only."""
    pos, _, _ = sim.get_state()
    counts, lists = sim.neighbours()
    L = sim.box[0]
    n = len(counts)
    species = sim.species
    rc = np.asarray(params["rcut"])
    sel = np.arange(0, n, max(1, n // sample))
    c, lst = counts[sel], lists[sel]
    rows = np.repeat(sel, c)
    cols = lst[np.arange(lst.shape[1])[None, :] < c[:, None]]
    d = pos[rows] - pos[cols]
    d -= L * np.round(d / L)
    r2 = (d * d).sum(1)
    inside = r2 < rc[species[rows], species[cols]] ** 2
    return counts.mean(), inside.sum() / len(sel)


def prepare(md, synth, n, seed, precision, device, use_graph=True, tpp=0):
    s = synth.ka_mixture(n=n, temperature=2.0, seed=seed)
    sim = md.System.from_synth(s, dt=0.001, precision=md.PRECISIONS[precision], sample_interval=100,
                               device=device, use_graph=use_graph, threads_per_particle=tpp)
    for _ in range(20):          # melt at T = 2
        sim.step(100)
        sim.rescale(2.0)
    for _ in range(20):          # quench to T = 0.5 by rescaling
        sim.step(100)
        sim.rescale(0.5)
    assert sim.sync() == md.MD_OK
    sim.observables()            # drop the preparation samples
    return s, sim


def time_iterations(torch, sim, nsteps_inner, k, flush, stream):
    """k timed md_step(nsteps_inner) calls, the L2 flushed before each; the
    device time of each call (CUDA events on the launching stream), in ms."""
    ms = []
    for _ in range(k):
        flush.fill_(1)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sim.step(nsteps_inner)
        e1.record(stream)
        ms.append((e0, e1))
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in ms]


def time_chunks(torch, sim, nsteps_inner, k, flush, stream):
    return sum(time_iterations(torch, sim, nsteps_inner, k, flush, stream))


def median_of_groups(iter_ms, groups=5):
    """The timed iterations split into `groups` consecutive groups: the median
    of the groups' mean times per iteration (ms), or None with fewer iterations."""
    if len(iter_ms) < groups:
        return None
    parts = np.array_split(np.asarray(iter_ms, dtype=np.float64), groups)
    return float(np.median([p.mean() for p in parts]))


def energy_drift(obs, n):
    """Least-squares slope of the total energy per particle per step, relative
    to |E/N|, over the recorded NVE samples."""
    if len(obs) < 3:
        return None, None
    e = (obs["e_pot"] + obs["e_kin"]) / n
    t = obs["step"].astype(np.float64)
    slope = np.polyfit(t - t[0], e, 1)[0]
    return float(slope / abs(e.mean())), float(np.abs(e - e[0]).max() / abs(e.mean()))


def run_ours(args, rank, world, local):
    import torch
    from paper_0912_3824_gb300 import build as b
    b.build()
    from paper_0912_3824_gb300 import md, synth

    torch.cuda.set_device(local)
    device = f"cuda:{local}"
    stream = torch.cuda.current_stream(device)
    s, sim = prepare(md, synth, args.n, 5 + rank, args.precision, device,
                     use_graph=not args.no_graph, tpp=args.tpp)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=device)
    # launch shape (lanes per particle), skin and list capacity from the autotuner, on
    # the prepared state; --no-tune keeps --tpp / --skin as given
    pos0, vel0, img0 = sim.get_state()
    base = md.make_params(s.params, 0.001, skin=args.skin, precision=md.PRECISIONS[args.precision],
                          sample_interval=100, use_graph=not args.no_graph, threads_per_particle=args.tpp,
                          check_interval=args.check, step_form=args.step_form, build_form=args.build_form)
    trials = None
    if not args.no_tune:
        from paper_0912_3824_gb300 import tune
        base, trials = tune.autotune(base, [s.n], [s.box], s.species, pos0, vel0, img0, device=device)
    sim.close()
    sim = md.System(base, [s.n], [s.box], s.species, pos0, vel0, img0, device=device)

    for _ in range(args.warmup):
        flush.fill_(1)
        sim.step(args.inner)
    assert sim.sync() == md.MD_OK
    sim.observables()
    info0 = sim.info()
    clocks = ClockSampler(local)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    # cudaProfilerStart/Stop bracket the timed region, so a profiler started
    # with profiling off (ncu --profile-from-start off) sees exactly its launches
    torch.cuda.profiler.start()
    iter_ms = time_iterations(torch, sim, args.inner, args.steps, flush, stream)
    total_ms = sum(iter_ms)
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    clk = clocks.stop()
    if world > 1:
        torch.distributed.barrier()
    status = sim.sync()
    info1 = sim.info()
    obs = sim.observables()[:, 0]
    drift, maxdev = energy_drift(obs, args.n)
    work = float(args.n) * args.inner * args.steps
    gathered = allgather_floats([work, total_ms / 1e3], world)
    value, tmax = aggregate([g[0] for g in gathered], [g[1] for g in gathered])
    launches = int(info1["kernel_launches"] - info0["kernel_launches"])
    rebuilds = int(info1["rebuilds"] - info0["rebuilds"])

    result = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": tmax * 1e3 / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        # the timed iterations in 5 consecutive groups: the median group, as particle-steps/s
        # of this rank, beside the spread of single iterations
        "repeats": {"groups": 5, "median_ms_per_step": median_of_groups(iter_ms),
                    "median_value": (float(args.n) * args.inner / (median_of_groups(iter_ms) * 1e-3)
                                     if median_of_groups(iter_ms) else None),
                    "min_ms_per_step": float(min(iter_ms)), "max_ms_per_step": float(max(iter_ms))},
        "dtype": {"mixed": "f32 pair math, f32x2 (double-single) state", "fp64": "f64", "fp32": "f32"}[args.precision],
        "data": "synthetic (seeded fcc lattice, melted and quenched on the GPU)",
        "config": {"workload": ka_workload(args.n),
                   "precision": args.precision, "md_steps_per_iteration": args.inner,
                   "l2": "flushed (256 MB write) between timed iterations",
                   "parallelism": f"replicas x{world} (no collective)",
                   "threads_per_particle": info1["threads_per_particle"],
                   "check_interval": info1["check_interval"],
                   "neigh_capacity": info1["neigh_capacity"], "skin": float(base.skin),
                   "epot": "every MD step (fused into the force loop; md_epot_series)",
                   "samples": "full observables every 100 MD steps",
                   "tuned": trials is not None},
        "clocks": clk, "gpu_launches": launches,
        "autotune": [{k: (round(v, 5) if isinstance(v, float) else v) for k, v in t.items()} for t in trials]
                    if trials else None,
        "md": {"rebuilds_in_timed_region": rebuilds, "status": md._status_name(status),
               "energy_drift_per_step_rel": drift, "energy_max_rel_dev": maxdev,
               "samples": int(len(obs))},
    }
    if args.no_extras or rank != 0:
        return result

    # ---- force kernel: live per-launch duration (stream launches + CUDA events) ----
    pos, vel, img = sim.get_state()
    p_nog = md.make_params(s.params, 0.001, skin=base.skin, precision=md.PRECISIONS[args.precision],
                           sample_interval=100, use_graph=False, threads_per_particle=base.threads_per_particle,
                           neigh_capacity=base.neigh_capacity)
    sim_k = md.System(p_nog, [s.n], [s.box], s.species, pos, vel, img, device=device)
    sim_k.step(32)
    info_a = sim_k.info()
    sim_k.step(320)
    info_b = sim_k.info()
    ev_ms = (info_b["step_ms"] - info_a["step_ms"]) / max(1, info_b["step_launches"] - info_a["step_launches"])
    # the step kernel's average duration inside the timed region (the CUDA-graph run),
    # from the device timer each launch reads at its first block start and last block end
    n_dev = info1["step_device_launches"] - info0["step_device_launches"]
    f_ms = (info1["step_device_ms"] - info0["step_device_ms"]) / max(1, n_dev)
    n_list, n_cut = list_statistics(sim_k, s.params)
    sim_k.close()
    flops = (FLOP_PER_ENTRY_METHOD * n_list + FLOP_PER_PAIR_METHOD * n_cut) * s.n
    flops_kernel = (FLOP_PER_ENTRY * n_list + FLOP_PER_PAIR * n_cut + FLOP_PER_UPDATE) * s.n
    sm_mhz = clk.get("sm_mhz") or 1.9e3
    peaks = alu_peaks(md, torch, device)
    peak_max = peaks["fp32_tflops"]
    result["roofline"] = {
        "bound": "alu", "kernel": f"k_step<{args.precision}, {info1['threads_per_particle']}, unsmoothed> "
                                  "(pair forces and energy + velocity-Verlet update)",
        "achieved": flops / (f_ms * 1e-3) / 1e12, "peak": peak_max, "unit": "TFLOP/s",
        "frac": flops / (f_ms * 1e-3) / 1e12 / peak_max,
        "flop_convention": f"{FLOP_PER_ENTRY_METHOD} per list entry + {FLOP_PER_PAIR_METHOD} per pair in the "
                           "cutoff (the method's count for mixed precision)",
        "kernel_count": {"flop_per_launch": flops_kernel, "tflops": flops_kernel / (f_ms * 1e-3) / 1e12,
                         "note": f"{FLOP_PER_ENTRY} per entry + {FLOP_PER_PAIR} per pair + {FLOP_PER_UPDATE} "
                                 "per particle (update), counted as this kernel computes"},
        "traffic": profiled_traffic(f"k_step<{md.PRECISIONS[args.precision]}, {info1['threads_per_particle']}, 0, "
                                    f"{1 if info1['step_form'] == 2 else 0}>", base.skin),
        "per_launch_ms": f_ms, "launches_timed": int(n_dev),
        "per_launch_ms_events": ev_ms,
        "timing": "per_launch_ms: device timer over the timed region (every k_step launch of the graph); "
                  "per_launch_ms_events: CUDA events around stream launches of the same kernel",
        "flop_per_launch": flops, "mean_list": float(n_list),
        "mean_in_cutoff": float(n_cut),
        "peak_note": "FP32 FMA peak measured on this GPU by md_fma_peak (FMA chains on every SM, CUDA "
                     "events); nominal beside it: SMs x 128 lanes x 2 flop x max clock",
        "peaks": peaks,
        "frac_of_nominal": flops / (f_ms * 1e-3) / 1e12 / peaks["fp32_nominal_tflops"],
        "frac_at_sampled_clock": flops / (f_ms * 1e-3) / (peaks["sms"] * 128 * 2 * sm_mhz * 1e6),
        "hbm_view": {"algorithmic_bytes_per_launch": float(s.n * (4 * n_list + 32 + 16 + 4)),
                     "achieved_gbs": s.n * (4 * n_list + 52) / (f_ms * 1e-3) / 1e9,
                     "peak_gbs": (measured_peaks() or {}).get("hbm_gbs", 6800.0)},
    }

    # ---- same workload in full FP64 on the same GPU ----
    p64 = md.make_params(s.params, 0.001, skin=args.skin, precision=md.MD_PREC_FP64, sample_interval=100)
    if not args.no_tune:
        p64, _ = tune.autotune(p64, [s.n], [s.box], s.species, pos, vel, img, device=device)
    sim64 = md.System(p64, [s.n], [s.box], s.species, pos, vel, img, device=device)
    sim64.step(args.inner)
    k64 = max(3, args.steps // 20)
    ms64 = time_chunks(torch, sim64, args.inner, k64, flush, stream)
    assert sim64.sync() == md.MD_OK
    sim64.close()
    v64 = s.n * args.inner * k64 / (ms64 / 1e3)
    result["vs_fp64"] = {"fp64_value": v64, "speedup": value / world / v64, "fp64_iterations": k64}

    # ---- end to end through the C ABI with host buffers ----
    ke = max(3, min(args.steps, 20))
    pos_h = np.ascontiguousarray(pos)
    vel_h = np.ascontiguousarray(vel)
    img_h = np.ascontiguousarray(img)
    sim.set_state(pos_h, vel_h, img_h)
    sim.step(args.inner)
    sim.observables()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    nrec = 0
    for _ in range(ke):
        sim.set_state(pos_h, vel_h, img_h)
        sim.step(args.inner)
        o = sim.observables()
        nrec += o.size
    torch.cuda.synchronize()
    t_e2e = time.perf_counter() - t0
    result["e2e"] = {"value": s.n * args.inner * ke / t_e2e, "unit": UNIT,
                     "h2d_bytes_per_step": int(pos_h.nbytes + vel_h.nbytes + img_h.nbytes),
                     "d2h_bytes_per_step": int(nrec * 120 // ke + 104), "iterations": ke,
                     "step": f"one timed iteration: state up from host memory, md_step({args.inner}), "
                             "observables back"}
    sim.close()

    # ---- CPU baseline: the FP64 oracle as it stands, on the host cores ----
    if world == 1:
        result["cpu_baseline"] = cpu_baseline(s, pos, vel, img)
    return result


def alu_peaks(md, torch, device):
    """CUDA-core arithmetic peaks of this GPU: measured (FMA chains, md_fma_peak)
    and nominal (SM count from the device properties x 128 FP32 lanes x 2 flop
    x the maximum SM clock nvidia-smi reports)."""
    props = torch.cuda.get_device_properties(device)
    sms = int(props.multi_processor_count)
    fp32, ms32 = md.md_fma_peak(md.MD_PREC_FP32, 2000)
    fp64, ms64 = md.md_fma_peak(md.MD_PREC_FP64, 200)
    max_mhz = None
    try:
        out = subprocess.run(["nvidia-smi", "-i", str(torch.cuda.current_device()), "--query-gpu=clocks.max.sm",
                              "--format=csv,noheader,nounits"], capture_output=True, text=True, timeout=20)
        max_mhz = float(out.stdout.strip().splitlines()[0])
    except (OSError, ValueError, IndexError, subprocess.TimeoutExpired):
        pass
    mhz = max_mhz or 2070.0
    return {"fp32_tflops": fp32, "fp64_tflops": fp64, "fp32_ms": ms32, "fp64_ms": ms64, "sms": sms,
            "max_sm_mhz": mhz, "fp32_nominal_tflops": sms * 128 * 2 * mhz * 1e6 / 1e12,
            "how": "md_fma_peak: 8 independent FMA chains per thread, 4 waves of 256-thread blocks on every SM, "
                   "fastest of 3 launches (CUDA events); FMA = 2 flop"}


def _oracle_worker(job):
    """One host process: the oracle as it stands advancing its own copy of the
    state by nsteps velocity-Verlet steps; returns its wall time."""
    params, box, species, pos, vel, img, dt, nsteps = job
    import oracle
    t0 = time.perf_counter()
    oracle.vv_run(params, box, species, pos, vel, img, dt, nsteps)
    return time.perf_counter() - t0


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_all_cores(s, pos, vel, img, dt, nsteps, cores):
    """The oracle on every host core: `cores` spawned processes (a fork after the
    first GPU call could hang), each advancing its own copy of the workload by
    nsteps steps, started together; returns the wall time of the slowest."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    job = (s.params, s.box, s.species, pos, vel, img, dt, nsteps)
    with ctx.Pool(cores) as pool:
        pool.map(_oracle_worker, [(s.params, s.box, s.species, pos, vel, img, dt, 1)] * cores)   # imports, warm
        t0 = time.perf_counter()
        pool.map(_oracle_worker, [job] * cores, chunksize=1)
        return time.perf_counter() - t0


def cpu_baseline(s, pos, vel, img, budget_s=15.0, dt=0.001, all_cores=True):
    """The FP64 oracle on the host: one thread, and (all_cores) one process per
    host core, each on its own copy of the state (a replica ensemble: the oracle
    itself is serial).  `value` is the all-core aggregate when measured."""
    import oracle
    oracle.build()
    t0 = time.perf_counter()
    oracle.vv_run(s.params, s.box, s.species, pos, vel, img, dt, 2)
    per = (time.perf_counter() - t0) / 3.0          # 3 force evaluations
    nsteps = max(2, int(budget_s / per))
    t0 = time.perf_counter()
    oracle.vv_run(s.params, s.box, s.species, pos, vel, img, dt, nsteps)
    el = time.perf_counter() - t0
    one = {"value": s.n * nsteps / el, "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": f"{nsteps} velocity-Verlet steps of the same N={s.n} state, FP64 cell-list "
                     f"oracle, single thread ({el:.1f} s)"}
    cores = host_cores()
    if not all_cores or cores < 2:
        return one
    k = max(2, nsteps // 2)
    wall = oracle_all_cores(s, pos, vel, img, dt, k, cores)
    return {"value": cores * s.n * k / wall, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{cores} host processes (one per core in the affinity mask), each advancing its own "
                      f"copy of the N={s.n} state by {k} velocity-Verlet steps with the FP64 cell-list oracle "
                      f"as it stands ({wall:.1f} s wall); aggregate particle-steps/s",
            "single_core": one}


# ---------------------------------------------------------------------------
# Further workloads (--workload ...): the other configurations of the method's
# evaluation.  Each prints one JSON line per case; none is the headline line.
# ---------------------------------------------------------------------------
def _gpu_setup(local):
    import torch
    from paper_0912_3824_gb300 import build as b
    b.build()
    from paper_0912_3824_gb300 import md, synth
    torch.cuda.set_device(local)
    device = f"cuda:{local}"
    stream = torch.cuda.current_stream(device)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=device)
    return torch, md, synth, device, stream, flush


def equilibrate(sim, t_melt, t_final, melt_blocks=20, final_blocks=20, block=100):
    """Melt the lattice at t_melt and bring the liquid to t_final, rescaling
    the velocities after every block of MD steps."""
    for _ in range(melt_blocks):
        sim.step(block)
        sim.rescale(t_melt)
    for _ in range(final_blocks):
        sim.step(block)
        sim.rescale(t_final)


def unwrapped(pos, img, box):
    return pos + img * box


def run_lj_sweep(args, local):
    """LJ fluid at rho = 0.8442, T = 1.0, dt = 0.005, skin 0.3, in the chosen
    precision, N from 4096 to 1048576: throughput against system size."""
    cases = [(n, 0.8442) for n in (args.sizes or [4096, 32768, 262144, 1048576])]
    return lj_cases(args, local, cases, "lj-sweep", temperature=1.0, dt=0.005, skin=0.3)


def run_e1(args, local):
    """The performance measurements of Sec. 3: LJ (r_c = 2.5) at T = 1.5,
    dt = 0.001, skin 0.5, N = 1372 ... 864000 (4 n^3) and densities 0.2 ... 1.2."""
    cases = [(n, rho) for rho in (args.densities or [0.2, 0.4, 0.8, 1.2])
             for n in (args.sizes or [1372, 10976, 87808, 864000])]
    return lj_cases(args, local, cases, "e1", **E1)


def lj_cases(args, local, cases, workload, temperature, dt, skin):
    torch, md, synth, device, stream, flush = _gpu_setup(local)
    peaks = alu_peaks(md, torch, device)
    hbm_peak = (measured_peaks() or {}).get("hbm_gbs", 6800.0)
    lines = []
    for n, rho in cases:
        s = synth.lj_fluid(n=n, density=rho, temperature=temperature, seed=3)
        sim = md.System.from_synth(s, dt=dt, skin=skin, precision=md.PRECISIONS[args.precision],
                                   sample_interval=100, device=device, threads_per_particle=args.tpp,
                                   use_graph=not args.no_graph, step_form=args.step_form,
                                   build_form=args.build_form)
        equilibrate(sim, max(1.5, temperature), temperature, melt_blocks=5, final_blocks=5)
        trials = None
        if not args.no_tune:
            # lanes per particle from the autotuner; the skin is the workload's own
            from paper_0912_3824_gb300 import tune
            pos0, vel0, img0 = sim.get_state()
            base = md.make_params(s.params, dt, skin=skin, precision=md.PRECISIONS[args.precision],
                                  sample_interval=100, threads_per_particle=args.tpp, use_graph=not args.no_graph,
                                  step_form=args.step_form, build_form=args.build_form)
            base, trials = tune.autotune(base, [s.n], [s.box], s.species, pos0, vel0, img0, device=device,
                                         skins=(skin,))
            sim.close()
            sim = md.System(base, [s.n], [s.box], s.species, pos0, vel0, img0, device=device)
        sim.step(args.inner)                       # warm-up, graph captured
        assert sim.sync() == md.MD_OK
        sim.observables()
        info0 = sim.info()
        clocks = ClockSampler(local)
        clocks.start()
        torch.cuda.profiler.start()          # (ncu --profile-from-start off sees the timed region)
        ms = time_chunks(torch, sim, args.inner, args.steps, flush, stream)
        torch.cuda.profiler.stop()
        clk = clocks.stop()
        status = sim.sync()
        info1 = sim.info()
        n_dev = info1["step_device_launches"] - info0["step_device_launches"]
        k_ms = (info1["step_device_ms"] - info0["step_device_ms"]) / max(1, n_dev)
        n_list, n_cut = list_statistics(sim, s.params)
        t_step = ms * 1e-3 / (args.inner * args.steps)
        # the method's count and the peak of the precision the pair loop runs in
        if args.precision == "mixed":
            flops = (FLOP_PER_ENTRY_METHOD * n_list + FLOP_PER_PAIR_METHOD * n_cut) * n
        else:
            flops = (FLOP_PER_ENTRY_PLAIN * n_list + FLOP_PER_PAIR_PLAIN * n_cut) * n
        alu_peak = peaks["fp64_tflops"] if args.precision == "fp64" else peaks["fp32_tflops"]
        hbm = n * (4 * n_list + 52 + 192)
        line = {"workload": workload,
                "config": f"LJ rho={rho} T={temperature} dt={dt} r_c=2.5 shifted skin {skin}, N={n}",
                "precision": args.precision, "n": n, "density": rho, "value": n / t_step, "unit": UNIT,
                "ns_per_particle_step": t_step / n * 1e9,
                "us_per_md_step": t_step * 1e6, "md_steps": args.inner * args.steps,
                "rebuilds": int(info1["rebuilds"] - info0["rebuilds"]), "status": md._status_name(status),
                "mean_list": float(n_list), "mean_in_cutoff": float(n_cut),
                "neigh_capacity": info1["neigh_capacity"], "threads_per_particle": info1["threads_per_particle"],
                "alu_tflops_whole_step": flops / t_step / 1e12,
                "hbm_algorithmic_gbs_whole_step": hbm / t_step / 1e9,
                "step_kernel_us": k_ms * 1e3,
                "step_kernel_alu_tflops": flops / (k_ms * 1e-3) / 1e12 if k_ms > 0 else None,
                "step_kernel_list_gbs": n * (4 * n_list + 52) / (k_ms * 1e-3) / 1e9 if k_ms > 0 else None,
                # roofline fractions of the step kernel: its algorithmic flops against the
                # measured FMA peak of its precision (FP64 for the FP64 mode, FP32 otherwise),
                # its algorithmic bytes (list + own state + the fused integrator's state
                # traffic) against the measured HBM copy rate
                "step_kernel_alu_frac": flops / (k_ms * 1e-3) / 1e12 / alu_peak if k_ms > 0 else None,
                "step_kernel_alu_peak": "fp64" if args.precision == "fp64" else "fp32",
                "step_kernel_hbm_frac": n * (4 * n_list + 52 + 192) / (k_ms * 1e-3) / 1e9 / hbm_peak
                if k_ms > 0 else None,
                "peaks": {"fp32_tflops": peaks["fp32_tflops"], "fp64_tflops": peaks["fp64_tflops"],
                          "hbm_gbs": hbm_peak},
                "clocks": clk,
                "autotune": [{k: (round(v, 5) if isinstance(v, float) else v) for k, v in t.items()}
                             for t in trials] if trials else None}
        if n <= 32768 and not args.no_extras:
            pos, vel, img = sim.get_state()
            line["cpu_baseline"] = cpu_baseline(s, pos, vel, img, budget_s=5.0, dt=dt, all_cores=False)
        sim.close()
        lines.append(line)
    return lines


def run_replicas(args, local):
    """256 Kob-Andersen replicas with N_r uniform in {500, ..., 8000} at
    rho = 1.2, T = 0.8: one handle holding every replica (one CUDA graph per
    md_step) against one handle per replica launched in a loop."""
    torch, md, synth, device, stream, flush = _gpu_setup(local)
    sizes = synth.ensemble_sizes(256, 500, 8000, seed=4)
    reps = [synth.ka_mixture(n=m, temperature=0.8, seed=4000 + r) for r, m in enumerate(sizes)]
    prec = md.PRECISIONS[args.precision]
    p = md.make_params(reps[0].params, 0.001, precision=prec, sample_interval=100,
                       threads_per_particle=args.tpp)
    cat = lambda f: np.concatenate([getattr(r, f) for r in reps])
    boxes = [r.box for r in reps]
    trials = None
    if not args.no_tune:
        # lanes per particle, skin and list capacity for the whole ensemble (one handle)
        from paper_0912_3824_gb300 import tune
        p, trials = tune.autotune(p, sizes, boxes, cat("species"), cat("pos"), cat("vel"), cat("image"),
                                  device=device, steps=200)
    one = md.System(p, sizes, boxes, cat("species"), cat("pos"), cat("vel"), cat("image"), device=device)
    loop = [md.System(p, [r.n], [r.box], r.species, r.pos, r.vel, r.image, device=device) for r in reps]
    total = int(sum(sizes))

    def time_loop(k):
        evs = []
        for _ in range(k):
            flush.fill_(1)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for h in loop:
                h.step(args.inner)
            e1.record(stream)
            evs.append((e0, e1))
        torch.cuda.synchronize()
        return sum(a.elapsed_time(b) for a, b in evs)

    for _ in range(2):                            # warm-up: graphs captured, lists built
        one.step(args.inner)
        for h in loop:
            h.step(args.inner)
    torch.cuda.synchronize()
    ms_one = time_chunks(torch, one, args.inner, args.steps, flush, stream)
    ms_loop = time_loop(args.steps)
    st = [one.sync()] + [h.sync() for h in loop]
    work = total * args.inner * args.steps
    line = {"workload": "replicas", "config": "256 KA replicas, N_r ~ U{500..8000} (seed 4), rho=1.2, T=0.8, "
                                              "dt=0.001, replica seeds 4000+r",
            "precision": args.precision, "total_particles": total, "unit": UNIT,
            "one_handle": {"value": work / (ms_one * 1e-3), "us_per_md_step": ms_one * 1e3 / (args.inner * args.steps)},
            "per_replica_loop": {"value": work / (ms_loop * 1e-3),
                                 "us_per_md_step": ms_loop * 1e3 / (args.inner * args.steps)},
            "speedup": ms_loop / ms_one, "md_steps": args.inner * args.steps,
            "threads_per_particle": int(p.threads_per_particle), "skin": float(p.skin),
            "neigh_capacity": int(p.neigh_capacity), "tuned": trials is not None,
            "autotune": [{k: (round(v, 5) if isinstance(v, float) else v) for k, v in t.items()} for t in trials]
                        if trials else None,
            "status": sorted({md._status_name(x) for x in st})}
    one.close()
    for h in loop:
        h.close()
    return [line]


def nve_run(md, torch, stream, sim, n, box, species, nsteps, lags, chunk=50000):
    """NVE segment: energy samples, momentum, A-particle MSD at the given lags
    (from the unwrapped positions) and the device time of the MD steps."""
    pos0, _, img0 = sim.get_state()
    r0 = unwrapped(pos0, img0, box)
    sel = species == 0
    marks = sorted({int(l) for l in lags if 0 < l <= nsteps} | {nsteps})
    done, ms, samples, msd = 0, 0.0, [], {}
    for m in marks:
        while done < m:
            k = min(chunk, m - done)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            sim.step(k)
            e1.record(stream)
            e1.synchronize()
            ms += e0.elapsed_time(e1)
            samples.append(sim.observables()[:, 0])
            done += k
        if m in lags:
            pos, _, img = sim.get_state()
            d = unwrapped(pos, img, box) - r0
            msd[str(m)] = float((d[sel] ** 2).sum(1).mean())
    obs = np.concatenate(samples)
    return obs, ms, msd


def run_drift(args, local):
    """Energy drift, momentum and MSD in FP32, mixed and FP64 from the same
    equilibrated state: LJ N=864 (dt 0.005), KA N=16384 at T=0.7 (two seeds)
    and KA N=65536 quenched to T=0.5 (rescaled every step for 10^4 steps)."""
    from paper_0912_3824_gb300 import synth
    M = args.md_steps
    cases = [("lj864", lambda: synth.lj_fluid(864, density=0.8442, temperature=0.722, seed=1), 0.005,
              None, min(M, 100000)),
             ("ka16384-s2", lambda: synth.ka_mixture(16384, temperature=2.0, seed=2), 0.001, (2.0, 0.7), M),
             ("ka16384-s3", lambda: synth.ka_mixture(16384, temperature=2.0, seed=3), 0.001, (2.0, 0.7), M),
             ("ka65536", lambda: synth.ka_mixture(65536, temperature=2.0, seed=5), 0.001, (2.0, 0.5), M)]
    return nve_cases(args, local, cases, "drift")


def run_longrun(args, local):
    """KA N=65536 quenched to T=0.5 (rescaled after every step for 10^4 steps),
    then NVE for --md-steps steps (FP64: --fp64-steps, by default 1/5 of that)
    in each of --precisions (mixed and FP64 by default), for each smoothing
    width of --smooth (the plain cut and h = 0.005 of Sec. 4 by default) at
    time step --dt (0.001 by default) and each of --seeds (5 by default): the
    energy drift per particle over a long run."""
    from paper_0912_3824_gb300 import synth
    cases = []
    dt = args.dt or KA_DT
    for sd in (args.seeds or [5]):
        for h in (args.smooth if args.smooth is not None else (0.0, 0.005)):
            params = synth.ka_params(smooth=h)
            cases.append((f"ka65536-h{h}-dt{dt}" + (f"-s{sd}" if sd != 5 else ""),
                          lambda params=params, sd=sd: synth.make_system(65536, 1.2, 2.0, sd, params),
                          dt, (2.0, 0.5), args.md_steps))
    emit = lambda ln: print(json.dumps(ln), flush=True)
    fp64_steps = args.fp64_steps if args.fp64_steps else max(1000, args.md_steps // 5)
    nve_cases(args, local, cases, "longrun", precisions=tuple(args.precisions or ("mixed", "fp64")),
              steps_of={"fp64": fp64_steps}, emit=emit)
    return []


def run_stats(args, local):
    """The long-run comparison against FP64 over independent runs: KA N=65536
    (per seed), melted and quenched to T=0.5 (rescaled after every step for
    10^4 steps), then --md-steps NVE steps in FP32, mixed and FP64 from the
    same quenched state.  One line per seed and precision as it completes,
    then the summary (mean and standard error over seeds; mixed and FP32
    against FP64)."""
    from paper_0912_3824_gb300 import synth
    seeds = args.seeds or [5, 6, 7, 8]
    precs = tuple(args.precisions or ("fp32", "mixed", "fp64"))
    cases = [(f"ka65536-s{sd}", lambda sd=sd: synth.ka_mixture(65536, temperature=2.0, seed=sd), KA_DT,
              (2.0, 0.5), args.md_steps) for sd in seeds]
    lags = sorted({int(round(10 ** (k / 2))) for k in range(2, 13)})     # 10, 32, 100, ... 10^6
    emit = lambda ln: print(json.dumps(ln), flush=True)
    lines = nve_cases(args, local, cases, "stats", precisions=precs, lags=lags, emit=emit)
    return [dict(workload="stats", **stats_summary(lines))]


def run_drift_floor(args, local):
    """What sets the FP64 energy drift: KA (--particles, 16384 by default here)
    in FP64 with the smoothing of Sec. 4 and with the plain cut, varying the
    time step (equal simulated time), the rebuild-check interval and the skin.
    Integrator error would scale with dt; missed pairs with the check interval
    and the skin; reduction rounding with neither."""
    from paper_0912_3824_gb300 import synth
    n = args.n if args.n != 65536 else 16384
    t_sim = args.md_steps * 0.001
    cases = []
    for h in (0.005, 0.0):
        params = synth.ka_params(smooth=h)
        mk = lambda params=params: synth.make_system(n, 1.2, 2.0, 5, params)
        for dt, extra in ((0.001, {}), (0.0005, {}), (0.001, {"check_interval": 1}),
                          (0.001, {"skin": 0.6})):
            tag = "-".join(f"{k}{v}" for k, v in extra.items()) or "base"
            cases.append((f"ka{n}-h{h}-dt{dt}-{tag}", mk, dt, (2.0, 0.5), int(round(t_sim / dt)), extra))
    precs = tuple(args.precisions or ("fp64",))
    emit = lambda ln: print(json.dumps(ln), flush=True)
    nve_cases(args, local, cases, "drift-floor", precisions=precs, lags=[10 ** 9], emit=emit)
    return []


def run_stability(args, local):
    """The stability protocol of Sec. 4: N = 10000 at rho = 0.75, T = 1.12,
    LJ (r_c = 2.5) and WCA, dt = 0.001 and 0.003, smoothing h = 0 and 0.005,
    each in FP32, mixed and FP64 from the same equilibrated state."""
    from paper_0912_3824_gb300 import synth
    cases = []
    st = STABILITY
    for pot in ("wca", "lj"):
        for h in st["smooth"]:
            for dt in st["dts"]:
                mk = synth.wca_params if pot == "wca" else synth.lj_params
                params = mk(smooth=h)
                cases.append((f"{pot}-h{h}-dt{dt}",
                               lambda params=params: synth.make_system(st["n"], st["density"], st["temperature"],
                                                                       12, params),
                               dt, (st["temperature"], st["temperature"]), args.md_steps))
    return nve_cases(args, local, cases, "stability")


def nve_cases(args, local, cases, workload, precisions=("fp32", "mixed", "fp64"), steps_of=None, lags=None,
              emit=None):
    """Each case: (name, make, dt, temps, nsteps[, extra make_params keywords]).
    One line per case and precision; `emit` (if given) receives each line as
    soon as it is measured."""
    torch, md, synth, device, stream, flush = _gpu_setup(local)
    lags = lags or [10 ** k for k in range(1, 8)]
    if args.cases:
        cases = [c for c in cases if c[0] in args.cases]
    lines = []
    for case in cases:
        name, make, dt, temps, nsteps = case[:5]
        extra = case[5] if len(case) > 5 else {}
        s = make()
        prep = md.System.from_synth(s, dt=dt, precision=md.MD_PREC_MIXED, sample_interval=100, device=device)
        if temps is not None:
            equilibrate(prep, temps[0], temps[1])
            if name.startswith("ka65536"):        # quench: rescale after every step
                for _ in range(10000):
                    prep.step(1)
                    prep.rescale(temps[1])
        assert prep.sync() == md.MD_OK
        pos, vel, img = prep.get_state()
        prep.close()
        for prec in precisions:
            nsteps_p = (steps_of or {}).get(prec, nsteps)
            p = md.make_params(s.params, dt, precision=md.PRECISIONS[prec], sample_interval=100,
                               step_form=0 if prec == "fp64" else getattr(args, "step_form", 0), **extra)
            sim = md.System(p, [s.n], [s.box], s.species, pos, vel, img, device=device)
            obs, ms, msd = nve_run(md, torch, stream, sim, s.n, s.box, s.species, nsteps_p, lags)
            status = sim.sync()
            info = sim.info()
            sim.close()
            slope, maxdev = energy_drift(obs, s.n)
            pmax = float(np.abs(obs["p"]).max()) / s.n
            lines.append({"workload": workload, "case": name, "precision": prec, "n": s.n, "dt": dt,
                          "smooth_h": float(s.params.get("smooth", 0.0)),
                          "md_steps": nsteps_p, "value": s.n * nsteps_p / (ms * 1e-3), "unit": UNIT,
                          "us_per_md_step": ms * 1e3 / nsteps_p,
                          "energy_drift_per_step_rel": slope,
                          "energy_drift_total_rel": None if slope is None else slope * nsteps_p,
                          "energy_max_rel_dev": maxdev, "max_abs_momentum_per_particle": pmax,
                          "e_per_particle": float((obs["e_pot"][0] + obs["e_kin"][0]) / s.n),
                          "msd_A": msd, "rebuilds": int(info["rebuilds"]),
                          "params": {k: (float(v) if isinstance(v, float) else v) for k, v in extra.items()},
                          "status": md._status_name(status)})
            if emit is not None:
                emit(lines[-1])
    return lines


def stats_summary(lines, reference="fp64"):
    """Across independent runs (one line per seed and precision): per precision
    the mean and standard error of the energy-drift slope, of the largest
    |P|/N and of the A-particle MSD at each lag; then each precision against
    the reference precision: z = (mean - mean_ref) / sqrt(se^2 + se_ref^2)
    per quantity, and whether |z| <= 3 for every MSD lag."""
    by = {}
    for ln in lines:
        by.setdefault(ln["precision"], []).append(ln)

    def ms(vals):
        v = np.asarray([x for x in vals if x is not None], dtype=np.float64)
        if v.size == 0:
            return None
        se = float(v.std(ddof=1) / np.sqrt(v.size)) if v.size > 1 else None
        return {"mean": float(v.mean()), "se": se, "n": int(v.size)}

    out = {}
    for prec, ls in by.items():
        lags = sorted({int(k) for ln in ls for k in ln["msd_A"]})
        out[prec] = {"drift_per_step": ms([ln["energy_drift_per_step_rel"] for ln in ls]),
                     "max_abs_momentum_per_particle": ms([ln["max_abs_momentum_per_particle"] for ln in ls]),
                     "msd_A": {str(l): ms([ln["msd_A"].get(str(l)) for ln in ls]) for l in lags},
                     "runs": len(ls)}

    def z(a, b):
        if a is None or b is None or a["se"] is None or b["se"] is None:
            return None
        den = math.sqrt(a["se"] ** 2 + b["se"] ** 2)
        return (a["mean"] - b["mean"]) / den if den > 0 else 0.0

    ref = out.get(reference)
    cmp = {}
    if ref is not None:
        for prec, st in out.items():
            if prec == reference:
                continue
            zs = {l: z(st["msd_A"].get(l), ref["msd_A"].get(l)) for l in ref["msd_A"]}
            cmp[prec] = {"z_msd_A": zs,
                         "msd_A_within_3se": all(v is not None and abs(v) <= 3.0 for v in zs.values()),
                         "z_drift": z(st["drift_per_step"], ref["drift_per_step"]),
                         "momentum_ratio": (st["max_abs_momentum_per_particle"]["mean"] /
                                            ref["max_abs_momentum_per_particle"]["mean"])}
    return {"summary": out, "against": reference, "comparison": cmp}


def ka_workload(n):
    """The headline workload's name, shared by both arms."""
    return (f"Kob-Andersen 80:20, N={n} per GPU, rho=1.2, T=0.5 after quench, dt=0.001, "
            "r_c=2.5 sigma_ab shifted, NVE")


def run_reference(args, rank, world):
    """The FP64 CPU oracle as the reference arm, on the host cores: one spawned
    process per core in the affinity mask, each advancing its own copy of the
    workload (the oracle is serial; the copies make it a replica ensemble);
    each timed step = one MD step of every copy.  The single-thread rate is
    reported beside."""
    if rank != 0:
        return None
    import oracle
    from paper_0912_3824_gb300 import synth
    oracle.build()
    s = synth.ka_mixture(n=args.n, temperature=0.5, seed=5)
    pos, vel, img = s.pos, s.vel, s.image
    pos, vel, img, _, _ = oracle.vv_run(s.params, s.box, s.species, pos, vel, img, 0.001, args.warmup)
    # one call for all K steps: the oracle's extra force evaluation at entry is amortised
    t0 = time.perf_counter()
    oracle.vv_run(s.params, s.box, s.species, pos, vel, img, 0.001, args.steps)
    dt1 = time.perf_counter() - t0
    one = s.n * args.steps / dt1
    cores = host_cores()
    wall = oracle_all_cores(s, pos, vel, img, 0.001, args.steps, cores) if cores > 1 else dt1
    value = cores * s.n * args.steps / wall
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": wall * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded fcc lattice at T=0.5: the oracle's cost per step hardly "
                    "depends on the melt and quench that the GPU arm runs first)",
            "config": {"workload": ka_workload(args.n), "precision": "fp64 (CPU oracle)",
                       "md_steps_per_iteration": 1},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{cores} host processes, each {args.steps} velocity-Verlet steps of "
                                       f"its own copy of the N={s.n} state in one oracle call ({wall:.1f} s "
                                       "wall); aggregate particle-steps/s",
                             "single_core": {"value": one, "cores": 1,
                                             "sample": f"{args.steps} steps, one thread ({dt1:.1f} s)"}},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main(argv=None):
    args = parse_args(argv)
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        backend = "gloo" if args.impl == "reference" else "nccl"
        if args.impl != "reference":
            import torch
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    if args.workload != "ka65536":
        if args.impl == "reference" or world > 1:
            raise SystemExit("--workload other than ka65536 runs our path on one GPU only")
        fn = {"lj-sweep": run_lj_sweep, "e1": run_e1, "replicas": run_replicas, "drift": run_drift,
              "stability": run_stability, "longrun": run_longrun, "stats": run_stats,
              "drift-floor": run_drift_floor}[args.workload]
        for line in fn(args, local):
            print(json.dumps(line), flush=True)
        return
    if args.impl == "reference":
        res = run_reference(args, rank, world)
    else:
        res = run_ours(args, rank, world, local)
    if rank == 0 and res is not None:
        print(json.dumps(res))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
