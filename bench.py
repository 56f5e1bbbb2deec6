"""Benchmark: pair-interactions per second of the fused force + Velocity-Verlet step.

Workload: the cold Gaussian bunch of N = 65536 macro-electrons (1e8 electrons,
w = 1525.88), sigma = 10 um per coordinate, softening 1 nm, dt = 1e-14 s; seeded,
synthetic.  One "step" is one time step of the whole hot path: the O(N^2) force sum
(FP32 pairs, FP64 fold) with the push fused into its epilogue.  Throughput counts
N^2 pair interactions per step.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Timing: W untimed warm-up steps, then K steps, each bracketed by CUDA events on the
library's stream with a 256 MiB L2-flush write before it (outside the events).  Under
torchrun each rank runs its own bunch (weak scaling, no data-path collective); rank 0
prints one JSON line with the max time over ranks.  ``--impl reference`` times the
FP64 CPU oracle instead, on bounded samples of the same workload.
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

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np

from paper_2502_10640_gb300 import workloads as wl

METRIC = "G pair-interactions/s & % FP32 peak; served p50/p99 latency at force rel-L2<=1e-5"
UNIT = "Gpair-interactions/s"
FLOP_PER_PAIR = 20          # counting convention for the FP32 roofline
WORKLOAD = wl.GAUSSIAN_65536


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--e2e-steps", type=int, default=20)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--variant", default=None,
                    help="run this force-kernel variant (by name) instead of autotuning")
    ap.add_argument("--split", type=int, default=0,
                    help="with --variant: j-split override (0 = the library's plan)")
    ap.add_argument("--batch-steps", type=int, default=8,
                    help="steps of the 64-bunch mix, batched and one bunch per launch (0 = skip)")
    ap.add_argument("--serve-requests", type=int, default=32,
                    help="requests of the bounded serving trace (0 = skip)")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the 2^20-particle and all-FP64 comparison measurements")
    ap.add_argument("--lattice-steps", type=int, default=2000,
                    help="steps of the paper's 16^3 lattice, resident and per-launch (0 = skip)")
    return ap.parse_args()


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


def profiled_traffic(variant: str, split: int):
    """DRAM bytes per force launch of this plan (kernel variant, j-split override) from the
    committed ncu record, or None if no capture of this plan exists or the kernel sources
    differ from the ones the captures were taken on."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "force_f32x2_gaussian65536_traffic.json")
    try:
        with open(path) as f:
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


def cpu_baseline(seconds: float, bunch=WORKLOAD):
    """The FP64 oracle on this host's cores: fields at a bounded sample of targets
    against all N sources (pair-interactions per second)."""
    import oracle
    pos = bunch.positions()
    n = bunch.n
    cores = os.cpu_count() or 1
    m = 256
    idx = np.arange(m, dtype=np.int64) * (n // m)
    t0 = time.perf_counter()
    oracle.fields_subset(pos, bunch.w, bunch.eps, idx)
    first = time.perf_counter() - t0
    rate = m * n / max(first, 1e-9)
    m2 = int(min(n, max(m, rate * seconds / n)))
    idx = np.linspace(0, n - 1, m2).astype(np.int64)
    t0 = time.perf_counter()
    oracle.fields_subset(pos, bunch.w, bunch.eps, idx)
    el = time.perf_counter() - t0
    return {"value": m2 * n / el / 1e9, "unit": UNIT, "cores": int(os.environ.get("OMP_NUM_THREADS", cores)),
            "kind": "oracle",
            "sample": f"FP64 oracle fields at {m2} of {n} particles against all {n} sources "
                      f"({m2 * n:.3e} pairs, {el:.1f} s)",
            "single_thread": single_thread_oracle(bunch)}


def single_thread_oracle(bunch, targets: int = 512):
    """The same oracle call on one host thread (a child process with OMP_NUM_THREADS=1):
    `targets` sampled particles against all sources."""
    import subprocess
    import sys
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


def bunch_key(bunch) -> str:
    for k, v in wl.WORKLOADS.items():
        if v is bunch:
            return k
    raise KeyError(bunch.name)


def run_extras(sms: int, peak_tflops: float):
    """Side measurements on the same GPU: the single-bunch force step at N = 2^20 (the
    size the FP32 target is stated at) and the all-FP64 path on the benchmark bunch."""
    import torch
    from paper_2502_10640_gb300 import capi
    out = {}
    b = wl.SPHERE_1M
    with capi.Simulation(b.n, b.w, b.dt, b.eps, tune="cache") as sim:
        sim.load(b.positions())
        sim.step(1)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        stream = torch.cuda.Stream()
        sim.set_option(capi.PP_OPT_STREAM, stream.cuda_stream)
        ev[0].record(stream)
        sim.step(3)
        ev[1].record(stream)
        torch.cuda.synchronize()
        sec = ev[0].elapsed_time(ev[1]) / 1e3 / 3
        pairs = float(b.n) ** 2 / sec
        out["sphere_2p20"] = {"workload": b.name, "pairs_per_s": pairs, "ms_per_step": sec * 1e3,
                              "frac_fp32_peak": FLOP_PER_PAIR * pairs / 1e12 / peak_tflops,
                              "kernel": (sim.tuned or {}).get("variant_name")}
    g = WORKLOAD
    with capi.Simulation(g.n, g.w, g.dt, g.eps, acc=capi.PP_ACC_FP64_FULL) as sim:
        sim.load(g.positions())
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sim.step(1)
        sec = time.perf_counter() - t0
        out["fp64_path"] = {"workload": g.name, "pairs_per_s": float(g.n) ** 2 / sec,
                            "ms_per_step": sec * 1e3,
                            "note": "FP64 pair math and accumulation, one step"}
    return out


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


def run_batched(steps: int):
    """The 64-bunch mix (N log-uniform 1024-131072): one persistent launch per step for
    all bunches, against the plain path that steps each bunch with its own launches."""
    import torch
    from paper_2502_10640_gb300 import capi
    mix = wl.batch_mix()
    pairs = float(sum(x.n ** 2 for x in mix)) * steps
    with capi.Batch(150 << 30, graph_block=0) as bt:
        for x in mix:
            bt.add(x.positions(), x.w, x.dt, x.eps)
        bt.step(1)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        bt.step(steps)
        t_batch = time.perf_counter() - t0
    sims = []
    try:
        for x in mix:
            s_ = capi.Simulation(x.n, x.w, x.dt, x.eps)
            s_.set_option(capi.PP_OPT_GRAPH_BLOCK, 0)
            s_.load(x.positions())
            sims.append(s_)
        for s_ in sims:
            s_.step(1)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(steps):
            for s_ in sims:
                s_.step(1)
        t_plain = time.perf_counter() - t0
    finally:
        for s_ in sims:
            s_.close()
    return {"workload": f"{len(mix)} cold bunches, N log-uniform 1024-131072 (sum N^2 = "
                        f"{pairs / steps:.3e} per step), Gaussian/sphere 50/50",
            "steps": steps, "unit": UNIT,
            "batched": pairs / t_batch / 1e9,
            "one_bunch_per_launch": pairs / t_plain / 1e9,
            "speedup": t_plain / t_batch,
            "timing": "host wall clock around the synchronous step calls"}


def run_serving(count: int):
    """Bounded serving trace: Poisson arrivals at 20 requests/s of uniform-sphere runs,
    N and step counts scaled down (x1/8 and x1/20) so the run takes seconds."""
    from paper_2502_10640_gb300 import serve
    trace = wl.serve_trace(count)
    reqs = serve.requests_from_trace(trace, n_scale=0.125, steps_scale=0.05)
    srv = serve.Server(150 << 30, block_steps=16)
    try:
        rep = srv.run(reqs)
    finally:
        srv.close()
    return {"trace": f"{count} requests, Poisson 20/s, N log-uniform 512-65536 (1/8 of "
                     f"4096-524288), steps 5-250 (1/20 of 100-5000), budget 150 GB",
            "completed": rep["completed"], "p50_latency_s": rep.get("p50_latency_s"),
            "p99_latency_s": rep.get("p99_latency_s"), "pairs_per_s": rep["pairs_per_s"],
            "unit_pairs": "pair-interactions/s", "wall_s": rep["wall_s"], "blocks": rep["blocks"]}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    b = WORKLOAD
    pos = b.positions()
    n = b.n
    m = 128                                            # targets per sampled step
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
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded cold Gaussian bunch)",
        "config": {"workload": b.name, "N": n, "w": b.w, "eps_m": b.eps, "dt_s": b.dt,
                   "sample_per_step": f"fields at {m} of {n} targets against all {n} sources"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"each step: FP64 oracle fields at {m} of {n} targets "
                                   f"against all {n} sources"},
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
    b = WORKLOAD
    seed = b.seed + 1000 * rank
    pos0 = wl.gaussian_bunch(b.n, b.scale, seed)
    n = b.n
    stream = torch.cuda.Stream(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    sim = capi.Simulation(n, b.w, b.dt, b.eps)
    sim.set_option(capi.PP_OPT_STREAM, stream.cuda_stream)
    sim.load(pos0)
    if args.variant:
        sim.set_option(capi.PP_OPT_VARIANT, capi.variants().index(args.variant))
        sim.set_option(capi.PP_OPT_SPLIT, args.split)
        tune = None
    else:
        tune = None if args.no_autotune else sim.autotune()     # set-up, not timed
    plan_variant = capi.variants()[sim.get_option(capi.PP_OPT_VARIANT)]
    plan_split = sim.get_option(capi.PP_OPT_SPLIT)
    for _ in range(args.warmup):
        sim.step(1)
    torch.cuda.synchronize(dev)

    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize(dev)
    with ClockSampler(local) as clocks:
        for k in range(args.steps):
            with torch.cuda.stream(stream):
                flush.fill_(float(k))                     # evict L2 (outside the events)
            starts[k].record(stream)
            sim.step(1)
            ends[k].record(stream)
        torch.cuda.synchronize(dev)
    if world > 1:
        torch.distributed.barrier()
    ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    total_s = sum(ms) / 1e3
    total_s = max_over_ranks(total_s)
    pairs = float(n) * n * args.steps * world
    value = pairs / total_s / 1e9

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
            for k in range(args.e2e_steps):
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
               "api": "pp_set_state(pinned host r,v,a) + pp_step(1) + pp_get_state(pinned host "
                      "r,v,a), PP_MEM_HOST_MAPPED",
               "copy_engine_value": rate(t_copy),
               "copy_engine_api": "the same calls with PP_MEM_HOST (copy engine through scratch)"}

    sim.close()
    batched = run_batched(args.batch_steps) if (args.batch_steps > 0 and world == 1) else None
    extras = None
    if not args.no_extras and world == 1:
        pk, _ = load_peaks()
        extras = run_extras(sms, fp32_peak_tflops(sms, float(pk.get("sm_max_mhz", 2070.0))))
    served = run_serving(args.serve_requests) if (args.serve_requests > 0 and world == 1) else None
    lattice = run_paper_lattice(args.lattice_steps) if (args.lattice_steps > 0 and world == 1) else None
    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return 0

    peaks, peak_src = load_peaks()
    csum = clocks.summary()
    max_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    peak = fp32_peak_tflops(sms, max_mhz)
    per_step_ms = 1e3 * total_s / args.steps
    achieved = FLOP_PER_PAIR * float(n) * n / (per_step_ms / 1e3) / 1e12
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": per_step_ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded cold Gaussian bunch)",
        "config": {"workload": b.name, "N": n, "w": b.w, "eps_m": b.eps, "dt_s": b.dt,
                   "precision": "FP32 pair math, FP64 per-particle fold, FP64 r/v/a",
                   "l2": "flushed before every timed step (256 MiB write)",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                   "pct_fp32_peak": 100.0 * achieved / peak,
                   "kernel": plan_variant,
                   "split": plan_split,
                   "autotuned": tune is not None},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": profiled_traffic(plan_variant, plan_split),
                     "note": f"{FLOP_PER_PAIR} flop per pair; peak = 2 x 128 FP32 lanes x {sms} SMs x "
                             f"{max_mhz:.0f} MHz ({'sm_max_mhz of measured peaks file' if peak_src == 'measured' else 'fallback clock'})"},
        "gpu_launches": args.steps,
        "e2e": e2e,
        "clocks": csum,
    }
    if extras:
        line.update(extras)
    if batched:
        line["batched"] = batched
    if served:
        line["serving"] = served
    if lattice:
        line["paper_lattice"] = lattice
    if not args.no_cpu_baseline and world == 1:
        line["cpu_baseline"] = cpu_baseline(args.cpu_seconds)
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
