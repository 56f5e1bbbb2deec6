"""Benchmark: pair-interactions per second of the fused force + Velocity-Verlet step.

Headline workload: the cold uniform sphere of N = 2^20 macro-electrons, R = 50 um,
Q = 1 nC (w = 5952.4), softening 5 nm, dt = 2e-14 s; seeded, synthetic.  One "step" is
one time step of the whole hot path: the O(N^2) force sum (FP32 pairs, FP64 fold) with
the push fused into its epilogue.  Throughput counts N^2 pair interactions per step.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Timing: W untimed warm-up steps, then K steps, each bracketed by CUDA events on the
library's stream with a 256 MiB L2-flush write before it (outside the events).  Under
torchrun each rank runs its own bunch (weak scaling, no data-path collective); rank 0
prints one JSON line with the max time over ranks.  ``--impl reference`` times the FP64
CPU oracle instead, on bounded samples of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np

from paper_2502_10640_gb300 import workloads as wl

METRIC = "G pair-interactions/s & % FP32 peak; served p50/p99 latency at force rel-L2<=1e-5"
UNIT = "Gpair-interactions/s"
FLOP_PER_PAIR = 20          # counting convention for the FP32 roofline
WORKLOAD = wl.SPHERE_1M     # the headline: the largest single-GPU configuration
SIDE_WORKLOAD = wl.GAUSSIAN_65536
L2_FLUSH_BYTES = 256 * 1024 * 1024
POSITIONS = {"auto": 2, "single": 0, "split": 1, "guarded": 3}   # pp_positions values


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="sphere1m", choices=sorted(wl.WORKLOADS),
                    help="the timed bunch (default: the N = 2^20 sphere; others for profiling)")
    ap.add_argument("--positions", default="auto", choices=sorted(POSITIONS),
                    help="staging of the timed bunch (default: the library's PP_POS_AUTO)")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--autotune", action="store_true",
                    help="autotune the headline bunch (a few minutes at N = 2^20) instead of "
                         "running the library's own plan")
    ap.add_argument("--variant", default=None,
                    help="run this force-kernel variant (by name) for the headline bunch")
    ap.add_argument("--split", type=int, default=0,
                    help="with --variant: j-split override (0 = the library's plan)")
    ap.add_argument("--side-steps", type=int, default=20,
                    help="timed steps of the N = 65536 Gaussian side figure (0 = skip)")
    ap.add_argument("--kahan-steps", type=int, default=3,
                    help="timed steps of the headline bunch with the compensated fold (0 = skip)")
    ap.add_argument("--batch-steps", type=int, default=16,
                    help="steps of the 64-bunch mix, batched and one bunch per launch (0 = skip)")
    ap.add_argument("--serve-requests", type=int, default=32,
                    help="requests of the bounded serving trace (0 = skip)")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the all-FP64 comparison measurement")
    ap.add_argument("--lattice-steps", type=int, default=2000,
                    help="steps of the paper's 16^3 lattice, resident and per-launch (0 = skip)")
    return ap.parse_args(argv)


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(x: float) -> float:
    """Maximum of a host scalar over all ranks (identity without torch.distributed)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return x
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" \
        else torch.device("cpu")
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f), "measured"
    return {"sm_max_mhz": 2070.0}, "fallback"


def bench_config(bunch, world: int) -> dict:
    """The `config` of the JSON line: the workload only (both arms print the same)."""
    return {"workload": bunch.name, "N": bunch.n, "w": bunch.w, "eps_m": bunch.eps,
            "dt_s": bunch.dt, "profile": bunch.profile, "scale_m": bunch.scale,
            "seed": bunch.seed, "steps_of_full_run": bunch.steps,
            "l2": "flushed before every timed step (256 MiB write)",
            "parallelism": f"replicas x{world}" if world > 1 else "single GPU"}


TRAFFIC_FILES = {"sphere1m": "force_f32x2_sphere1m_traffic.json",
                 "gaussian65536": "force_f32x2_gaussian65536_traffic.json"}


def profiled_traffic(workload_key: str, variant: str, split: int):
    """DRAM bytes per force launch of this plan (kernel variant, j-split override) on this
    workload from the committed ncu record, or None if no capture of this plan exists or
    the kernel sources differ from the ones the captures were taken on."""
    name = TRAFFIC_FILES.get(workload_key)
    if name is None:
        return None
    try:
        with open(os.path.join(ROOT, "profiles", name)) as f:
            rec = json.load(f)
        h = hashlib.sha256()
        for src in rec["sources"]:
            with open(os.path.join(ROOT, src), "rb") as f:
                h.update(f.read())
    except (OSError, ValueError, KeyError):
        return None
    if h.hexdigest() != rec["sources_sha256"]:
        return None
    for r in rec["records"]:
        if r["variant"] == variant and int(r["split"]) == int(split):
            return r["dram_bytes_read_per_launch"] + r["dram_bytes_write_per_launch"]
    return None


def fp32_peak_tflops(sms: int, mhz: float) -> float:
    """FP32 FMA pipe: 128 lanes per SM, 2 flop per FMA."""
    return 2.0 * 128 * sms * mhz * 1e6 / 1e12


class ClockSampler:
    """Samples SM clocks and throttle reasons with nvidia-smi while running."""

    QUERY = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.thread = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, ValueError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.thread.join(timeout=2)
        return False

    def summary(self):
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax = float(parts[1])
            except ValueError:
                continue
            for nm, val in zip(names, parts[4:8]):
                if val.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def bunch_key(bunch) -> str:
    for k, v in wl.WORKLOADS.items():
        if v is bunch:
            return k
    raise KeyError(bunch.name)


def sample_targets(n: int, m: int) -> np.ndarray:
    """m evenly spread target indices of an n-particle bunch."""
    return np.linspace(0, n - 1, m).astype(np.int64)


def cpu_baseline(seconds: float, bunch=WORKLOAD):
    """The FP64 oracle on this host's cores: fields at a bounded sample of targets against
    all N sources (pair-interactions per second), sized to about `seconds` of work."""
    import oracle
    pos = bunch.positions()
    n = bunch.n
    cores = os.cpu_count() or 1
    m = 512
    t0 = time.perf_counter()
    oracle.fields_subset(pos, bunch.w, bunch.eps, sample_targets(n, m))
    first = time.perf_counter() - t0
    rate = m * n / max(first, 1e-9)
    m2 = int(min(n, max(m, rate * seconds / n)))
    t0 = time.perf_counter()
    oracle.fields_subset(pos, bunch.w, bunch.eps, sample_targets(n, m2))
    el = time.perf_counter() - t0
    value = m2 * n / el / 1e9
    return {"value": value, "unit": UNIT,
            "cores": int(os.environ.get("OMP_NUM_THREADS", cores)), "kind": "oracle",
            "sample": f"FP64 oracle fields at {m2} of {n} particles against all {n} sources "
                      f"({m2 * n:.3e} pairs, {el:.1f} s)",
            "extrapolated_s_per_step": float(n) * n / (value * 1e9),
            "extrapolation": "one full step = N^2 pairs at the sampled rate (labelled "
                             "extrapolation: the oracle cannot run a full step of this size "
                             "in the bench's time)",
            "single_thread": single_thread_oracle(bunch)}


def single_thread_oracle(bunch, targets: int = 256):
    """The same oracle call on one host thread (a child process with OMP_NUM_THREADS=1):
    `targets` sampled particles against all sources."""
    code = ("import sys, time, numpy as np; sys.path.insert(0, sys.argv[1]); import oracle;"
            "from paper_2502_10640_gb300 import workloads as wl;"
            f"b = wl.WORKLOADS[{bunch_key(bunch)!r}]; pos = b.positions();"
            f"idx = np.linspace(0, b.n - 1, {targets}).astype(np.int64);"
            "oracle.fields_subset(pos, b.w, b.eps, idx[:8]);"
            "t0 = time.perf_counter(); oracle.fields_subset(pos, b.w, b.eps, idx);"
            "print(time.perf_counter() - t0)")
    env = dict(os.environ, OMP_NUM_THREADS="1")
    try:
        out = subprocess.run([sys.executable, "-c", code, ROOT], env=env, capture_output=True,
                             text=True, timeout=300, check=True)
        el = float(out.stdout.strip().splitlines()[-1])
    except (subprocess.SubprocessError, ValueError, IndexError) as e:
        return {"error": str(e)[:200]}
    return {"value": targets * bunch.n / el / 1e9, "unit": UNIT, "cores": 1,
            "sample": f"{targets} of {bunch.n} particles against all {bunch.n} sources "
                      f"({targets * bunch.n:.3e} pairs, {el:.2f} s)"}


def timed_steps(sim, stream, flush, steps: int):
    """Per-step CUDA-event times (ms) of `steps` single steps on `stream`, each after an
    L2-flush write outside the events."""
    import torch
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    for k in range(steps):
        with torch.cuda.stream(stream):
            flush.fill_(float(k))
        starts[k].record(stream)
        sim.step(1)
        ends[k].record(stream)
    torch.cuda.synchronize()
    return [s.elapsed_time(e) for s, e in zip(starts, ends)]


def plan_of(sim) -> dict:
    from paper_2502_10640_gb300 import capi
    return {"kernel": capi.variants()[sim.get_option(capi.PP_OPT_VARIANT)],
            "split": sim.get_option(capi.PP_OPT_SPLIT),
            "positions": {capi.PP_POS_SINGLE: "single", capi.PP_POS_SPLIT: "hi/lo",
                          capi.PP_POS_GUARDED: "guarded"}[sim.get_option(capi.PP_OPT_POSITIONS)],
            "staging_check": sim.staging_check(),
            "positions_chosen_by": "PP_POS_AUTO" if sim.get_option(capi.PP_OPT_POSITIONS_AUTO)
            else "explicit",
            "launches_per_step": sim.get_option(capi.PP_OPT_LAUNCHES_PER_PASS)}


def roofline_record(bunch, ms_per_step: float, peak: float, plan: dict, max_mhz: float,
                    sms: int, peak_src: str) -> dict:
    achieved = FLOP_PER_PAIR * float(bunch.n) ** 2 / (ms_per_step / 1e3) / 1e12
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak,
            "traffic": profiled_traffic(bunch_key(bunch), plan["kernel"], plan["split"]),
            "note": f"{FLOP_PER_PAIR} flop per pair, N^2 pairs per step; duration: CUDA events "
                    f"around one step ({plan['launches_per_step']} launches: the force kernel"
                    f"{' and the spatial sort of the tile-box guard' if plan['launches_per_step'] > 1 else ''}); "
                    f"peak = 2 x 128 FP32 lanes x {sms} SMs x {max_mhz:.0f} MHz "
                    f"({'sm_max_mhz of the measured peaks file' if peak_src == 'measured' else 'fallback clock'})"}


def run_side_figure(steps: int, stream, flush, peak: float, max_mhz: float, sms: int,
                    peak_src: str):
    """The N = 65536 Gaussian bunch (the second stated configuration) in the same timing
    discipline as the headline."""
    from paper_2502_10640_gb300 import capi
    b = SIDE_WORKLOAD
    with capi.Simulation(b.n, b.w, b.dt, b.eps) as sim:   # the library's own plan
        sim.set_option(capi.PP_OPT_STREAM, stream.cuda_stream)
        sim.load(b.positions())
        plan = plan_of(sim)
        sim.step(3)
        ms = timed_steps(sim, stream, flush, steps)
    per = sum(ms) / len(ms)
    return {"workload": b.name, "N": b.n, "steps": steps, "ms_per_step": per,
            "pairs_per_s": float(b.n) ** 2 / (per / 1e3), "plan": plan,
            "roofline": roofline_record(b, per, peak, plan, max_mhz, sms, peak_src)}


def run_kahan(steps: int, stream, flush, peak: float):
    """The headline bunch with the compensated FP32 fold (PP_ACC_KAHAN) beside the FP64
    fold of the headline line."""
    from paper_2502_10640_gb300 import capi
    b = WORKLOAD
    with capi.Simulation(b.n, b.w, b.dt, b.eps, acc=capi.PP_ACC_KAHAN) as sim:
        sim.set_option(capi.PP_OPT_STREAM, stream.cuda_stream)
        sim.load(b.positions())
        plan = plan_of(sim)
        sim.step(1)
        ms = timed_steps(sim, stream, flush, steps)
    per = sum(ms) / len(ms)
    pairs = float(b.n) ** 2 / (per / 1e3)
    return {"workload": b.name, "steps": steps, "ms_per_step": per, "pairs_per_s": pairs,
            "frac_fp32_peak": FLOP_PER_PAIR * pairs / 1e12 / peak, "plan": plan,
            "fold": "compensated FP32 pair per component (TwoSum), converted to FP64 once"}


def run_fp64_path():
    """The all-FP64 comparison path on the N = 65536 bunch, one step."""
    import torch
    from paper_2502_10640_gb300 import capi
    g = SIDE_WORKLOAD
    with capi.Simulation(g.n, g.w, g.dt, g.eps, acc=capi.PP_ACC_FP64_FULL) as sim:
        sim.load(g.positions())
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sim.step(1)
        sec = time.perf_counter() - t0
    return {"workload": g.name, "pairs_per_s": float(g.n) ** 2 / sec, "ms_per_step": sec * 1e3,
            "note": "FP64 pair math and accumulation, one step (host clock)"}


def run_paper_lattice(steps: int):
    """The paper's own workload (Sec. 2.1): the 16^3 cube lattice, eps = 0, dt = 1e-13 s,
    stepped with the library's default small-N path (the resident kernel: all steps of
    one call in one cooperative launch), against per-launch kernels with CUDA graphs."""
    import torch
    from paper_2502_10640_gb300 import capi
    b = wl.PAPER_LATTICE
    out = {"workload": b.name, "steps": steps, "paper_run_steps": b.steps}
    for label, mode in (("resident", capi.PP_RESIDENT_AUTO), ("per_launch", capi.PP_RESIDENT_OFF)):
        with capi.Simulation(b.n, b.w, b.dt, b.eps) as sim:
            sim.set_option(capi.PP_OPT_RESIDENT, mode)
            sim.load(b.positions())
            sim.step(16)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            sim.step(steps)
            sec = (time.perf_counter() - t0) / steps
            out[f"{label}_us_per_step"] = sec * 1e6
            if label == "resident":
                out["resident_active"] = bool(sim.get_option(capi.PP_OPT_RESIDENT_ACTIVE))
                out["paper_run_s"] = sec * b.steps
                out["pairs_per_s"] = float(b.n) ** 2 / sec
    out["timing"] = "host wall clock around one synchronous pp_step call"
    return out


def run_batched(steps: int, stream):
    """The 64-bunch mix (N log-uniform 1024-131072): one persistent launch per step for
    all bunches (autotuned kernel shape), against the plain path that steps each bunch
    with its own launch.  Both run on one stream bracketed by CUDA events, so the plain
    path's gaps between launches count."""
    import torch
    from paper_2502_10640_gb300 import capi
    mix = wl.batch_mix()
    pairs = float(sum(x.n ** 2 for x in mix)) * steps
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    with capi.Batch(150 << 30) as bt:
        bt.set_option(capi.PP_OPT_STREAM, stream.cuda_stream)
        slots = [bt.add(x.positions(), x.w, x.dt, x.eps) for x in mix]
        modes = [bt.get_option(capi.PP_OPT_POSITIONS, s) for s in slots]
        tune = bt.autotune()
        bt.step(2)
        torch.cuda.synchronize()
        ev[0].record(stream)
        bt.step(steps)
        ev[1].record(stream)
        torch.cuda.synchronize()
    t_batch = ev[0].elapsed_time(ev[1]) / 1e3
    sims = []
    try:
        for x in mix:
            s_ = capi.Simulation(x.n, x.w, x.dt, x.eps)
            s_.set_option(capi.PP_OPT_GRAPH_BLOCK, 0)
            s_.set_option(capi.PP_OPT_STREAM, stream.cuda_stream)
            s_.load(x.positions())
            sims.append(s_)
        for s_ in sims:
            s_.step(1)
        torch.cuda.synchronize()
        ev[2].record(stream)
        for _ in range(steps):
            for s_ in sims:
                s_.step(1)
        ev[3].record(stream)
        torch.cuda.synchronize()
    finally:
        for s_ in sims:
            s_.close()
    t_plain = ev[2].elapsed_time(ev[3]) / 1e3
    return {"workload": f"{len(mix)} cold bunches, N log-uniform 1024-131072 (sum N^2 = "
                        f"{pairs / steps:.3e} per step), Gaussian/sphere 50/50, eps = 1e-4 R",
            "steps": steps, "unit": UNIT,
            "batched": pairs / t_batch / 1e9,
            "one_bunch_per_launch": pairs / t_plain / 1e9,
            "speedup": t_plain / t_batch,
            "bunch_staging": {"single": modes.count(capi.PP_POS_SINGLE),
                              "guarded": modes.count(capi.PP_POS_GUARDED),
                              "hi/lo": modes.count(capi.PP_POS_SPLIT)},
            "batch_shape": tune["shape_name"],
            "timing": "CUDA events on the shared stream around all steps of each path "
                      "(the plain path's host gaps between its synchronous calls included)"}


def run_serving(count: int, rate: float = 20.0):
    """Bounded serving trace: Poisson arrivals of uniform-sphere runs with N as specified
    (4096-524288) and step counts scaled by 1/30 so that the trace finishes in about a
    minute.  At the specified 20 requests/s the GPU is saturated (latency is mostly
    queueing); a lower rate shows service latency."""
    from paper_2502_10640_gb300 import serve
    trace = wl.serve_trace(count, rate=rate)
    reqs = serve.requests_from_trace(trace, n_scale=1.0, steps_scale=1.0 / 30)
    srv = serve.Server(150 << 30, block_steps=16)
    try:
        rep = srv.run(reqs)
    finally:
        srv.close()
    return {"trace": f"{count} requests, Poisson {rate:g}/s, N log-uniform 4096-524288 (as "
                     f"specified), steps 3-167 (1/30 of 100-5000), budget 150 GB",
            "arrival_rate_per_s": rate,
            "n_scale": 1.0, "steps_scale": 1.0 / 30,
            "completed": rep["completed"], "p50_latency_s": rep.get("p50_latency_s"),
            "p99_latency_s": rep.get("p99_latency_s"), "pairs_per_s": rep["pairs_per_s"],
            "unit_pairs": "pair-interactions/s", "wall_s": rep["wall_s"], "blocks": rep["blocks"],
            "mean_queueing_s": rep.get("mean_queueing_s")}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    b = wl.WORKLOADS[args.workload]
    pos = b.positions()
    n = b.n
    m = 256                                            # targets per sampled step
    stride = n // m
    for w in range(args.warmup):
        oracle.fields_subset(pos, b.w, b.eps, np.arange(m, dtype=np.int64) * stride + w % stride)
    t = 0.0
    for k in range(args.steps):
        idx = np.arange(m, dtype=np.int64) * stride + (k % stride)
        t0 = time.perf_counter()
        oracle.fields_subset(pos, b.w, b.eps, idx)
        t += time.perf_counter() - t0
    pairs = args.steps * m * n
    value = pairs / t / 1e9
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    sample = f"each step: FP64 oracle fields at {m} of {n} targets against all {n} sources"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": f"synthetic (seeded cold {b.profile})",
        "config": bench_config(b, world),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import torch
    from paper_2502_10640_gb300 import capi

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    capi.load()
    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count
    peaks, peak_src = load_peaks()
    max_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    peak = fp32_peak_tflops(sms, max_mhz)
    b = wl.WORKLOADS[args.workload]
    pos0 = wl.Bunch(b.name, b.n, b.w, b.eps, b.dt, b.steps, b.profile, b.scale,
                    b.seed + 1000 * rank).positions()
    n = b.n
    stream = torch.cuda.Stream(dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    sim = capi.Simulation(n, b.w, b.dt, b.eps, tune="cache" if args.autotune else None,
                          positions=POSITIONS[args.positions])
    sim.set_option(capi.PP_OPT_STREAM, stream.cuda_stream)
    sim.load(pos0)                       # the staging decision (PP_POS_AUTO) is set-up
    if args.variant:
        sim.set_option(capi.PP_OPT_VARIANT, capi.variants().index(args.variant))
        sim.set_option(capi.PP_OPT_SPLIT, args.split)
    plan = plan_of(sim)
    plan["autotuned"] = bool(args.autotune)
    for _ in range(args.warmup):
        sim.step(1)
    torch.cuda.synchronize(dev)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize(dev)
    with ClockSampler(local) as clocks:
        ms = timed_steps(sim, stream, flush, args.steps)
    if world > 1:
        torch.distributed.barrier()
    total_s = max_over_ranks(sum(ms) / 1e3)
    value = float(n) * n * args.steps * world / total_s / 1e9
    per_step_ms = 1e3 * total_s / args.steps

    # end to end through the public API with pinned host buffers
    e2e = None
    if args.e2e_steps > 0:
        # pinned host buffers: as torch tensors the binding passes them as
        # PP_MEM_HOST_MAPPED (the kernels read and write them over the CPU-GPU link);
        # as numpy views of the same memory, as PP_MEM_HOST (copy engine + scratch)
        pin = [torch.empty((n, 3), dtype=torch.float64, pin_memory=True) for _ in range(3)]
        hp, hv, ha = (x.numpy() for x in pin)
        p, v, a, step, frame = sim.state()
        hp[:], hv[:], ha[:] = p, v, a

        def e2e_run(bufs):
            nonlocal step
            t = 0.0
            for _ in range(args.e2e_steps):
                torch.cuda.synchronize(dev)
                t0 = time.perf_counter()
                sim.set_state(*bufs, step, frame)
                sim.step(1)
                capi.pp_get_state(sim.ctx, *bufs)
                t += time.perf_counter() - t0
                step += 1
            return max_over_ranks(t)

        t_copy = e2e_run((hp, hv, ha))
        t_e2e = e2e_run(pin)
        rate = lambda t: float(n) * n * args.e2e_steps * world / t / 1e9
        e2e = {"value": rate(t_e2e), "unit": UNIT,
               "h2d_bytes_per_step": 3 * n * 3 * 8, "d2h_bytes_per_step": 3 * n * 3 * 8,
               "steps": args.e2e_steps,
               "api": "pp_set_state(pinned host r,v,a) + pp_step(1) + pp_get_state(pinned host "
                      "r,v,a), PP_MEM_HOST_MAPPED; host clock, synchronised",
               "copy_engine_value": rate(t_copy),
               "copy_engine_api": "the same calls with PP_MEM_HOST (copy engine through scratch)"}
    sim.close()

    extras = {}
    if world == 1:
        if args.kahan_steps > 0:
            extras["kahan_fold"] = run_kahan(args.kahan_steps, stream, flush, peak)
        if args.side_steps > 0:
            extras["gaussian_65536"] = run_side_figure(args.side_steps, stream, flush, peak,
                                                       max_mhz, sms, peak_src)
        if not args.no_extras:
            extras["fp64_path"] = run_fp64_path()
        if args.batch_steps > 0:
            extras["batched"] = run_batched(args.batch_steps, stream)
        if args.serve_requests > 0:
            extras["serving"] = run_serving(args.serve_requests)
            # the first 8 requests at 0.25/s offer about 0.75 of what the GPU serves:
            # latency without a standing backlog
            extras["serving_unsaturated"] = run_serving(min(8, args.serve_requests), rate=0.25)
        if args.lattice_steps > 0:
            extras["paper_lattice"] = run_paper_lattice(args.lattice_steps)
    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return 0

    roof = roofline_record(b, per_step_ms, peak, plan, max_mhz, sms, peak_src)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": per_step_ms,
        "step_ms": {"median": float(np.median(ms)), "min": float(min(ms)), "max": float(max(ms)),
                    "timing": "CUDA events around each timed step (this rank)"},
        "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": f"synthetic (seeded cold {b.profile})",
        "config": bench_config(b, world),
        "precision": "FP32 pair math, FP64 per-particle fold, FP64 r/v/a",
        "plan": plan,
        "pct_fp32_peak": 100.0 * roof["frac"],
        "roofline": roof,
        "gpu_launches": args.steps * plan["launches_per_step"],
        "e2e": e2e,
        "clocks": clocks.summary(),
    }
    line.update(extras)
    if not args.no_cpu_baseline and world == 1:
        line["cpu_baseline"] = cpu_baseline(args.cpu_seconds, b)
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
